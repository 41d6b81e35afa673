// Narrow planar complex products on the tensor cores (tcgen05.mma kind::tf32, split
// precision): C = alpha (op(A1) B1 [+ A2 B2]) + beta C with n <= 64 columns, the block
// products of the butterfly levels (Sec. 3, Eq. 3.3: U, R, B, W, V blocks times blocks of
// vectors) and of the solve.
//
// The product is computed transposed, so that the 64 right-hand sides fill the MMA's M = 128
// rows with both planes: with X = op-free B (k x n, row-major) and W = op(A) (m x k),
//   D (128 x m) = [Xr^T; Xi^T] Wr^T + [-Xi^T; Xr^T] Wi^T,
// rows 0..63 of D are (Wr Xr - Wi Xi)^T = Cr^T and rows 64..127 are (Wr Xi + Wi Xr)^T = Ci^T:
// one TMEM accumulator holds the whole complex result.  Shared memory holds X as the 192-row
// stack [Xr^T; Xi^T; -Xr^T]: the first operand is rows 0..127, the second rows 64..191 with
// the MMA's negate-A bit.  Every operand is split into hi = tf32(x) and lo = x - hi, and each
// real product is hi*hi + hi*lo + lo*hi (six MMAs per K step of 8), close to FP32 accuracy.
//
// Persistent CTAs (two per SM, 8 warps each) walk their share of the (product, 96-row tile)
// list as one stream of 16-wide K chunks: each chunk is loaded into registers one chunk ahead,
// split and written by whole 8 x 4 core matrices (conflict-free) into one of two shared
// memory slots in the canonical no-swizzle K-major layout, and thread 0 issues its MMAs and
// commits them to the slot's mbarrier, which frees the slot.  A tile's result alternates
// between two TMEM accumulators; its epilogue runs after the next tile's first MMAs are
// issued (so the tensor core works meanwhile), reads TMEM with tcgen05.ld (lane = right-hand
// side) and writes C rows with consecutive lanes on consecutive columns.  Every wait is
// bounded: on expiry the kernel records status 2, stops issuing work, drains and frees TMEM.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mf {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_BK = 16;                        // K elements per chunk
constexpr int TC_GRP = (TC_BK / 4) * 128;        // bytes per 8-row group of a tile (4 core matrices)
constexpr int TC_XTILE = (192 / 8) * TC_GRP;     // [Xr; Xi; -Xr]: 12 KB per hi / lo
constexpr int TC_ROWS = 96;                      // rows of W (columns of D) per tile
constexpr int TC_WTILE = (TC_ROWS / 8) * TC_GRP; // 96 rows of W: 6 KB per plane and hi / lo
constexpr int TC_SLOT = 2 * TC_XTILE + 4 * TC_WTILE;
constexpr int TC_SLOTS = 2;
constexpr int TC_SMEM = TC_SLOTS * TC_SLOT + 1024 + 128;   // two CTAs per SM
constexpr uint32_t TC_TMEM_COLS = 256;           // two accumulators of up to 128 columns
constexpr int TC_XBLK = (64 / 8) * (TC_BK / 4);  // core matrices of one X plane chunk: 32
constexpr int TC_MAXBLK = TC_XBLK + (TC_ROWS / 8) * (TC_BK / 4);
constexpr int TC_PER_WARP = (TC_MAXBLK + TC_WARPS - 1) / TC_WARPS;   // 10

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// byte offset of element (r, k) of a canonical no-swizzle K-major tile with 16-wide K chunks
__device__ __forceinline__ uint32_t cano(int r, int k) {
  return (uint32_t)((r >> 3) * TC_GRP + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = TC_GRP;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}
// instruction descriptor: D f32, A and B tf32 (K-major), M = 128, N = n
__device__ __forceinline__ uint32_t idesc(int n, int neg_a) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)neg_a << 13) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}
// hi = x rounded to the 10 explicit mantissa bits of TF32 (round half away from zero, low 13 bits
// cleared explicitly, so that the MMA reads hi exactly), lo = x - hi (exact in FP32)
__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  const uint32_t b = __float_as_uint(x);
  hi = __uint_as_float((b + 0x1000u) & 0xFFFFE000u);
  lo = x - hi;
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long spins) {
  for (long long i = 0; i < spins; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

// Where chunk c of tile t reads from: term (0: A/B, 1: A2/B2), K offset inside the term, K of the term.
struct Chunk {
  int t = 0, c = 0;   // tile index in the launch, chunk within the tile
};

__device__ __forceinline__ int tile_chunks(const GemmDesc<float>& d) {
  const int k1 = d.k1 > 0 ? d.k1 : d.k;
  return (k1 + TC_BK - 1) / TC_BK + (d.k1 > 0 ? (d.k - k1 + TC_BK - 1) / TC_BK : 0);
}

// Per-lane register copy of one chunk: up to TC_PER_WARP core matrices, real and imaginary value
struct Regs {
  float re[TC_PER_WARP], im[TC_PER_WARP];
};

// Load chunk ch into registers: core matrix b of the chunk (b < TC_XBLK: X, else W rows), lane
// -> (row 8 g + lane / 4, k 4 kg + lane % 4).  Out-of-range elements are zero.
__device__ __forceinline__ void load_chunk(Regs& R, const GemmDesc<float>* descs, const GemmTile* tiles, Chunk ch,
                                           int warp, int lane) {
  const GemmTile tl = tiles[ch.t];
  const GemmDesc<float>& d = descs[tl.desc];
  const int k1 = d.k1 > 0 ? d.k1 : d.k;
  const int nk1 = (k1 + TC_BK - 1) / TC_BK;
  const bool second = d.k1 > 0 && ch.c >= nk1;
  const int kt = second ? d.k - k1 : k1;                       // K of the term
  const int kc = (second ? ch.c - nk1 : ch.c) * TC_BK;         // chunk start inside the term
  const PMat<float> A = second ? d.A2 : d.A, B = second ? d.B2 : d.B;
  const int m0 = tl.tm * TC_ROWS;
  const int rows = min(TC_ROWS, d.m - m0);
  const int nwb = ((rows + 15) & ~15) / 8 * (TC_BK / 4);
  const int r8 = lane >> 2, k4 = lane & 3;
#pragma unroll
  for (int i = 0; i < TC_PER_WARP; ++i) {
    const int b = warp + TC_WARPS * i;
    float vr = 0.f, vi = 0.f;
    if (b < TC_XBLK) {
      const int col = (b >> 2) * 8 + r8, k = kc + (b & 3) * 4 + k4;   // X: 8 column groups x 4 k groups
      if (col < d.n && k < kt) {
        const float* p = B.re + (int64_t)k * B.ld + col;
        vr = __ldg(p);
        vi = __ldg(p + B.plane);
      }
    } else if (b - TC_XBLK < nwb) {
      const int bw = b - TC_XBLK;
      const int r = (bw >> 2) * 8 + r8, k = kc + (bw & 3) * 4 + k4;
      if (r < rows && k < kt) {
        const float* p = d.transA ? A.re + (int64_t)k * A.ld + m0 + r : A.re + (int64_t)(m0 + r) * A.ld + k;
        vr = __ldg(p);
        vi = __ldg(p + A.plane);
      }
    }
    R.re[i] = vr;
    R.im[i] = vi;
  }
}

// Split the registers into hi / lo and write them to slot s (conflict-free: a warp writes whole
// core matrices)
__device__ __forceinline__ void store_chunk(const Regs& R, unsigned char* slot, int nwb, int warp, int lane) {
  const int r8 = lane >> 2, k4 = lane & 3;
#pragma unroll
  for (int i = 0; i < TC_PER_WARP; ++i) {
    const int b = warp + TC_WARPS * i;
    float rh, rl, ih, il;
    split(R.re[i], rh, rl);
    split(R.im[i], ih, il);
    if (b < TC_XBLK) {
      const int col = (b >> 2) * 8 + r8, k = (b & 3) * 4 + k4;
      float* xh = reinterpret_cast<float*>(slot);
      float* xl = reinterpret_cast<float*>(slot + TC_XTILE);
      const uint32_t o0 = cano(col, k) >> 2, o1 = cano(64 + col, k) >> 2, o2 = cano(128 + col, k) >> 2;
      xh[o0] = rh;
      xl[o0] = rl;
      xh[o1] = ih;
      xl[o1] = il;
      xh[o2] = -rh;
      xl[o2] = -rl;
    } else if (b - TC_XBLK < nwb) {
      const int bw = b - TC_XBLK;
      const int r = (bw >> 2) * 8 + r8, k = (bw & 3) * 4 + k4;
      const uint32_t o = cano(r, k) >> 2;
      float* w = reinterpret_cast<float*>(slot + 2 * TC_XTILE);
      w[o] = rh;
      w[o + TC_WTILE / 4] = rl;
      w[o + 2 * TC_WTILE / 4] = ih;
      w[o + 3 * TC_WTILE / 4] = il;
    }
  }
}

// C rows of tile t from TMEM accumulator acc (D columns = rows of the tile, lanes = right-hand sides)
__device__ __forceinline__ void epilogue(const GemmDesc<float>* descs, const GemmTile* tiles, int t, uint32_t acc,
                                         int warp, int lane) {
  const GemmTile tl = tiles[t];
  const GemmDesc<float>& d = descs[tl.desc];
  const int m0 = tl.tm * TC_ROWS;
  const int rows = min(TC_ROWS, d.m - m0);
  const int nt = (rows + 15) & ~15;
  const int q = (warp & 3) * 32 + lane;       // TMEM lane = row of D
  const int col = q & 63;                     // right-hand side
  float* C = d.C.re + (q >= 64 ? d.C.plane : 0);
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int half = nt / 2;                    // columns of D per warp group (a multiple of 8)
  const int c_begin = (warp >> 2) * half, c_end = c_begin + half;
#pragma unroll 1
  for (int c0 = c_begin; c0 < c_end; c0 += 8) {
    uint32_t v[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(acc + lane_base + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (col < d.n) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int r = c0 + e;
        if (r < rows) {
          const int64_t off = (int64_t)(m0 + r) * d.C.ld + col;
          float val = d.alpha * __uint_as_float(v[e]);
          if (d.beta != 0.f) val += d.beta * C[off];
          C[off] = val;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 2) k_gemm_nrhs_tc(const GemmDesc<float>* __restrict__ descs,
                                                                 const GemmTile* __restrict__ tiles, int ntiles,
                                                                 int32_t* status, long long spins) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if ((int)blockIdx.x >= ntiles) return;
  const uint32_t sbase = (smem_u32(smem) + 1023u) & ~1023u;
  unsigned char* sgen = smem + (sbase - smem_u32(smem));
  const uint32_t bar0 = sbase + TC_SLOTS * TC_SLOT;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sgen + TC_SLOTS * TC_SLOT + 64);
  if (tid == 0) {
    for (int s = 0; s <= TC_SLOTS; ++s)   // one per slot and a spare that nothing arrives at
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar0 + 8 * s), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  if (spins <= kProbeWaitLimit)   // expiry test: the spare barrier never completes
    ok = __syncthreads_and(mbar_wait(bar0 + 8 * TC_SLOTS, 0u, spins) ? 1 : 0) != 0;
  Chunk cur;
  cur.t = ok ? (int)blockIdx.x : ntiles;   // after an expired test wait the CTA issues no work
  cur.c = 0;
  Regs ra, rb;
  if (cur.t < ntiles) load_chunk(ra, descs, tiles, cur, warp, lane);
  long long g = 0;      // chunks issued by this CTA
  int j = 0;            // tiles completed (MMAs issued) by this CTA
  int pend_t = -1;      // tile whose epilogue is pending, its accumulator and last chunk
  uint32_t pend_acc = 0;
  long long pend_g = 0;
#pragma unroll 1
  while (cur.t < ntiles) {
    const GemmTile tl = tiles[cur.t];
    const GemmDesc<float>& d = descs[tl.desc];
    const int nk = tile_chunks(d);
    const int rows = min(TC_ROWS, d.m - tl.tm * TC_ROWS);
    const int nt = (rows + 15) & ~15;
    const int slot = (int)(g % TC_SLOTS);
    unsigned char* sp = sgen + slot * TC_SLOT;
    const uint32_t sa = sbase + slot * TC_SLOT;
    // the slot is free once the MMAs of its previous chunk (g - TC_SLOTS) are complete
    if (g >= TC_SLOTS) ok = mbar_wait(bar0 + 8 * slot, (uint32_t)(((g / TC_SLOTS) - 1) & 1), spins);
    if (ok) store_chunk(ra, sp, nt / 8 * (TC_BK / 4), warp, lane);
    Chunk nx = cur;
    if (++nx.c == nk) {
      nx.c = 0;
      nx.t += gridDim.x;
    }
    if (ok && nx.t < ntiles) load_chunk(rb, descs, tiles, nx, warp, lane);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (__syncthreads_or(ok ? 0 : 1)) {
      ok = false;
      break;
    }
    const uint32_t acc_tm = tmem + (uint32_t)((j & 1) * 128);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t id_p = idesc(nt, 0), id_n = idesc(nt, 1);
      const uint32_t xh = sa, xl = sa + TC_XTILE;
      const uint32_t x2 = 8 * TC_GRP;   // rows 64.. of the X stack
      const uint32_t wrh = sa + 2 * TC_XTILE, wrl = wrh + TC_WTILE, wih = wrh + 2 * TC_WTILE, wil = wrh + 3 * TC_WTILE;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        const uint32_t ko = kk * 256;
        const uint32_t acc = (cur.c > 0 || kk > 0) ? 1u : 0u;
        mma(acc_tm, sdesc(xh + ko), sdesc(wrh + ko), id_p, acc);
        mma(acc_tm, sdesc(xh + ko), sdesc(wrl + ko), id_p, 1u);
        mma(acc_tm, sdesc(xl + ko), sdesc(wrh + ko), id_p, 1u);
        mma(acc_tm, sdesc(xh + x2 + ko), sdesc(wih + ko), id_n, 1u);
        mma(acc_tm, sdesc(xh + x2 + ko), sdesc(wil + ko), id_n, 1u);
        mma(acc_tm, sdesc(xl + x2 + ko), sdesc(wih + ko), id_n, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar0 + 8 * slot)
                   : "memory");
    }
    ++g;
    // the previous tile's epilogue, while the tensor core works on this chunk
    if (cur.c == 0 && pend_t >= 0) {
      ok = mbar_wait(bar0 + 8 * (int)(pend_g % TC_SLOTS), (uint32_t)((pend_g / TC_SLOTS) & 1), spins);
      if (__syncthreads_or(ok ? 0 : 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      epilogue(descs, tiles, pend_t, pend_acc, warp, lane);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
      pend_t = -1;
    }
    if (nx.t != cur.t) {   // last chunk of the tile: its epilogue waits for the next tile's first chunk
      pend_t = cur.t;
      pend_acc = acc_tm;
      pend_g = g - 1;
      ++j;
    }
    ra = rb;
    cur = nx;
  }
  if (ok && pend_t >= 0) {
    ok = mbar_wait(bar0 + 8 * (int)(pend_g % TC_SLOTS), (uint32_t)((pend_g / TC_SLOTS) & 1), spins);
    if (!__syncthreads_or(ok ? 0 : 1)) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      epilogue(descs, tiles, pend_t, pend_acc, warp, lane);
    } else {
      ok = false;
    }
  }
  // drain: every MMA this CTA issued has completed before TMEM is released (with the default
  // limit even after an expired wait, so that no MMA can still write the columns being freed)
  if (tid == 0 && g > 0) {
    const int slot = (int)((g - 1) % TC_SLOTS);
    if (!mbar_wait(bar0 + 8 * slot, (uint32_t)(((g - 1) / TC_SLOTS) & 1), kDefaultWaitLimit)) ok = false;
  }
  if (!ok && status) atomicExch(status, 2);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
}

}  // namespace

int gemm_nrhs_tc_rows() { return TC_ROWS; }

bool gemm_nrhs_tc_ok(const GemmDesc<float>& d) { return d.n <= 64 && d.transB == 0 && d.m > 0 && d.k > 0; }

void launch_gemm_nrhs_tc(const GemmDesc<float>* d_desc, const GemmTile* d_tiles, int ntiles, int32_t* status,
                         cudaStream_t st) {
  if (ntiles <= 0) return;
  static PerDeviceOnce attr;
  attr([] { cudaFuncSetAttribute(k_gemm_nrhs_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM); });
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ntiles < 2 * sms ? ntiles : 2 * sms;   // two CTAs per SM
  count_launches(1);
  k_gemm_nrhs_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(d_desc, d_tiles, ntiles, status, wait_limit());
}

}  // namespace mf
