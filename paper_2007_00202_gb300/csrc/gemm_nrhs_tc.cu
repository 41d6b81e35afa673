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
// Persistent CTAs (one per SM) walk their share of the (product, 96-row tile) list as one
// stream of 16-wide K chunks, with two warp roles:
//  * 8 producer warps.  Global loads are asynchronous (cp.async, zero-filled outside the
//    operands) into per-thread raw staging, TC_NRAW - 1 chunks ahead of use, so that HBM latency
//    is covered across tile boundaries.  The tiles' records and product descriptors are fetched
//    into shared-memory rings (16-byte cp.async) several tiles ahead, so that no global load
//    sits on the producers' path.  Each thread splits the elements it staged itself (no barrier
//    between copy and split) and writes them by whole 8 x 4 core matrices (conflict-free) into
//    one of two shared memory slots in the canonical no-swizzle K-major layout, then meet the
//    MMA warp at a named barrier.
//  * 1 MMA warp: after the barrier of chunk g, while the producers stage chunk g + 1, one lane
//    issues chunk g's MMAs and commits them to the slot's mbarrier, and after a tile's last
//    chunk to the accumulator's "full" mbarrier, beside the tile's epilogue record; it joins
//    the next barrier only once those MMAs are complete, so that the producers, who refill the
//    slot after that barrier, never wait on it themselves.  Tiles rotate over four TMEM
//    accumulators.
//  * 4 epilogue warps (TMEM lanes 0-127, lane = right-hand side and plane) wait for a tile's
//    accumulator, read it with tcgen05.ld 32 rows at a time, write C rows with consecutive lanes
//    on consecutive columns and release the accumulator ("empty" mbarrier) while later tiles are
//    computed.
// Every wait is bounded: on expiry the kernel records status 2, stops issuing work, drains its
// copies and MMAs and frees TMEM.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mf {

namespace {

constexpr int TC_PROD = 256;                     // producer threads (8 warps)
constexpr int TC_EPI = 128;                      // epilogue threads (4 warps)
constexpr int TC_MMA_WARP = (TC_PROD + TC_EPI) / 32;   // warp 12 issues the MMAs
constexpr int TC_THREADS = TC_PROD + TC_EPI + 32;
constexpr int TC_SYNC = TC_PROD + 32;            // producers and the MMA warp meet once per chunk
constexpr int TC_WARPS = TC_PROD / 32;           // producer warps
constexpr int TC_BK = 16;                        // K elements per chunk
constexpr int TC_GRP = (TC_BK / 4) * 128;        // bytes per 8-row group of a tile (4 core matrices)
constexpr int TC_XTILE = (192 / 8) * TC_GRP;     // [Xr; Xi; -Xr]: 12 KB per hi / lo
constexpr int TC_ROWS = 96;                      // rows of W (columns of D) per tile
constexpr int TC_WTILE = (TC_ROWS / 8) * TC_GRP; // 96 rows of W: 6 KB per plane and hi / lo
constexpr int TC_SLOT = 2 * TC_XTILE + 4 * TC_WTILE;
constexpr int TC_SLOTS = 2;
constexpr int TC_NACC = 4;                       // TMEM accumulators of up to 128 columns
constexpr uint32_t TC_TMEM_COLS = 128 * TC_NACC;
constexpr int TC_XBLK = (64 / 8) * (TC_BK / 4);  // core matrices of one X plane chunk: 32
constexpr int TC_MAXBLK = TC_XBLK + (TC_ROWS / 8) * (TC_BK / 4);
constexpr int TC_PER_WARP = (TC_MAXBLK + TC_WARPS - 1) / TC_WARPS;   // 10
constexpr int TC_NRAW = 6;                       // raw staging stages (copies run 5 chunks ahead)
constexpr int TC_RAW = 2 * TC_PER_WARP * TC_PROD * 4;   // bytes of one raw stage: 20 KB
constexpr int TC_DESC_BYTES = (int)sizeof(GemmDesc<float>);
constexpr int TC_TRING = 32, TC_TAHEAD = 16;     // tile records: ring size, fetch distance (tiles)
constexpr int TC_DRING = 16, TC_DAHEAD = 8;      // descriptors: ring size, fetch distance (tiles)
constexpr int TC_NBAR = TC_SLOTS + 2 * TC_NACC + 1;   // slots, full[], empty[], spare
constexpr int TC_OFF_RAW = TC_SLOTS * TC_SLOT;
constexpr int TC_OFF_DESC = TC_OFF_RAW + TC_NRAW * TC_RAW;
constexpr int TC_OFF_TILE = TC_OFF_DESC + TC_DRING * TC_DESC_BYTES;
constexpr int TC_OFF_EREC = TC_OFF_TILE + TC_TRING * 16;   // one epilogue record per accumulator
constexpr int TC_OFF_BAR = TC_OFF_EREC + TC_NACC * 48;
constexpr int TC_OFF_MISC = TC_OFF_BAR + 8 * TC_NBAR;
constexpr int TC_SMEM = TC_OFF_MISC + 16 + 1024;   // 1024: alignment of the slots
static_assert(TC_DESC_BYTES % 16 == 0 && TC_DESC_BYTES / 16 <= 31, "descriptor copies are 16-byte pieces");
static_assert(sizeof(GemmTile) == 16, "a tile record is one 16-byte piece");
static_assert(TC_OFF_DESC % 16 == 0 && TC_OFF_TILE % 16 == 0 && TC_OFF_EREC % 16 == 0 && TC_OFF_BAR % 8 == 0,
              "ring alignment");
static_assert(TC_SMEM <= 232448, "one CTA per SM");
// the copy cursor is at most TC_NRAW - 1 tiles ahead of the consumer: every ring holds the tiles
// from the consumer's to the furthest fetched
static_assert(TC_DRING >= TC_DAHEAD + TC_NRAW && TC_TRING >= TC_TAHEAD + TC_NRAW, "record rings too small");
// a record fetched when the copy cursor enters a tile is visible TC_NRAW iterations later
static_assert(TC_DAHEAD > TC_NRAW && TC_TAHEAD - TC_DAHEAD > TC_NRAW, "records fetched too late");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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
// Bounded wait that suspends the thread in the barrier (try_wait with a time hint of 1 us)
// instead of polling, so that the waiting warp leaves its issue slots to the producers; a
// suspended try counts as 64 polls of the limit, so the wait ends after about spins / 64 us.  It
// also gives up when another role has recorded a failure.
__device__ __forceinline__ bool mbar_try_suspend(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(1000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, long long spins,
                                                   const volatile int* abort) {
  const long long tries = spins > 64 ? spins >> 6 : 1;
  for (long long i = 0; i < tries; ++i) {
    if (mbar_try_suspend(bar, parity)) return true;
    if (*abort) return false;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
// barrier of the producer threads and the MMA warp (named barrier 1, TC_SYNC threads) that also
// ORs a flag over them
__device__ __forceinline__ bool chunk_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(TC_SYNC)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

// Position of the copy or consume cursor: tile t of the launch (the i-th of this CTA), chunk c.
struct Cursor {
  int t = 0, i = 0, c = 0;
};

// chunks of a tile; at least one, so that every cursor advances (a product with k = 0 runs one
// zero-filled chunk and writes beta C)
__device__ __forceinline__ int tile_chunks(const GemmDesc<float>& d) {
  const int k1 = d.k1 > 0 ? d.k1 : d.k;
  const int nk = (k1 + TC_BK - 1) / TC_BK + (d.k1 > 0 ? (d.k - k1 + TC_BK - 1) / TC_BK : 0);
  return nk > 0 ? nk : 1;
}

__device__ __forceinline__ void advance(Cursor& cu, const GemmDesc<float>* sd) {
  if (++cu.c == tile_chunks(sd[cu.i % TC_DRING])) {
    cu.c = 0;
    cu.t += gridDim.x;
    ++cu.i;
  }
}

// When the copy cursor enters its i-th tile, warp 1 fetches (into this iteration's copy group)
// the tile record of the (i + TC_TAHEAD)-th tile (lane 0) and the descriptor of the
// (i + TC_DAHEAD)-th tile (lanes 1..), whose tile record arrived TC_TAHEAD - TC_DAHEAD tiles ago.
__device__ __forceinline__ void fetch_records(int i, int ntiles, const GemmDesc<float>* descs, const GemmTile* tiles,
                                              uint32_t sdesc_u, uint32_t stile_u, const GemmTile* stile, int lane) {
  const int t1 = (int)blockIdx.x + (i + TC_TAHEAD) * (int)gridDim.x;
  if (lane == 0 && t1 < ntiles) cp16(stile_u + ((i + TC_TAHEAD) % TC_TRING) * 16, tiles + t1);
  const int t2 = (int)blockIdx.x + (i + TC_DAHEAD) * (int)gridDim.x;
  if (lane >= 1 && lane <= TC_DESC_BYTES / 16 && t2 < ntiles) {
    const int di = stile[(i + TC_DAHEAD) % TC_TRING].desc;
    cp16(sdesc_u + ((i + TC_DAHEAD) % TC_DRING) * TC_DESC_BYTES + (lane - 1) * 16,
         reinterpret_cast<const char*>(descs + di) + (lane - 1) * 16);
  }
}

// Asynchronous copy of chunk c of a tile into raw stage `raw` (shared address), d and tl the
// tile's descriptor and record (shared memory).  Thread (warp, lane) takes K index
// kq = 4 (warp % 4) + lane % 4 of the chunk and the 8-row groups g0 + 2 i (g0 = warp / 4):
// values i = 0..3 are X columns 8 (g0 + 2 i) + lane / 4, values i = 4..9 are W rows
// 8 (g0 + 2 (i - 4)) + lane / 4 (row groups of the tile only).  Value i goes to floats
// (2 i + plane) * TC_PROD + tid.  Elements outside the operands are zero-filled (source size 0,
// source address a valid dummy).  Does not commit.
__device__ __forceinline__ void copy_chunk(uint32_t raw, const GemmDesc<float>& d, const GemmTile tl, int c,
                                           const void* dummy, int warp, int lane, int tid) {
  const int k1 = d.k1 > 0 ? d.k1 : d.k;
  const int nk1 = (k1 + TC_BK - 1) / TC_BK;
  const bool second = d.k1 > 0 && c >= nk1;
  const int kt = second ? d.k - k1 : k1;                       // K of the term
  const int kc = (second ? c - nk1 : c) * TC_BK;               // chunk start inside the term
  const PMat<float> A = second ? d.A2 : d.A, B = second ? d.B2 : d.B;
  const int m0 = tl.tm * TC_ROWS;
  const int rows = min(TC_ROWS, d.m - m0);
  const int ngw = (rows + 15) / 16 * 2;                       // 8-row groups of W in the tile
  const int n = d.n;
  const int r8 = lane >> 2, g0 = warp >> 2;
  const int k = kc + (warp & 3) * 4 + (lane & 3);
  const bool kin = k < kt;
  const float* fdummy = static_cast<const float*>(dummy);
  const uint32_t dst0 = raw + (uint32_t)(tid * 4);
  {
    const float* px = B.re + (int64_t)(kin ? k : 0) * B.ld + 8 * g0 + r8;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool v = kin && 8 * (g0 + 2 * i) + r8 < n;
      const float* p = v ? px + 16 * i : fdummy;
      const uint32_t bytes = v ? 4u : 0u;
      const uint32_t dst = dst0 + (uint32_t)((2 * i) * TC_PROD * 4);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(p), "r"(bytes) : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst + TC_PROD * 4), "l"(v ? p + B.plane : p),
                   "r"(bytes)
                   : "memory");
    }
  }
  {
    const int r0 = 8 * g0 + r8;
    const int64_t step = d.transA ? 16 : 16 * A.ld;
    const float* pw = d.transA ? A.re + (int64_t)(kin ? k : 0) * A.ld + m0 + r0
                               : A.re + (int64_t)(m0 + (r0 < rows ? r0 : 0)) * A.ld + (kin ? k : 0);
#pragma unroll
    for (int j = 0; j < TC_PER_WARP - 4; ++j) {
      if (g0 + 2 * j >= ngw) continue;   // no element of this chunk: the raw value is never read
      const bool v = kin && r0 + 16 * j < rows;
      const float* p = v ? pw + step * j : fdummy;
      const uint32_t bytes = v ? 4u : 0u;
      const uint32_t dst = dst0 + (uint32_t)((2 * (4 + j)) * TC_PROD * 4);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(p), "r"(bytes) : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst + TC_PROD * 4), "l"(v ? p + A.plane : p),
                   "r"(bytes)
                   : "memory");
    }
  }
}

// Split this thread's staged values of a chunk into hi / lo and write them to slot s, at the
// positions copy_chunk gave them (conflict-free: a warp writes whole core matrices).  Element
// (r, k) of a canonical no-swizzle K-major tile with 16-wide K chunks sits at byte
// (r / 8) TC_GRP + (k / 4) 128 + (r % 8) 16 + (k % 4) 4.
__device__ __forceinline__ void store_chunk(const float* raw, unsigned char* slot, int ngw, int warp, int lane,
                                            int tid) {
  const int g0 = warp >> 2;
  const uint32_t base = (uint32_t)(g0 * TC_GRP + (warp & 3) * 128 + (lane >> 2) * 16 + (lane & 3) * 4) >> 2;
  float* xh = reinterpret_cast<float*>(slot);
  float* xl = reinterpret_cast<float*>(slot + TC_XTILE);
  float* w = reinterpret_cast<float*>(slot + 2 * TC_XTILE);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float rh, rl, ih, il;
    split(raw[(2 * i) * TC_PROD + tid], rh, rl);
    split(raw[(2 * i + 1) * TC_PROD + tid], ih, il);
    const uint32_t o0 = base + (uint32_t)(2 * i * TC_GRP / 4);   // rows col, 64 + col, 128 + col
    const uint32_t o1 = o0 + 8 * TC_GRP / 4, o2 = o0 + 16 * TC_GRP / 4;
    xh[o0] = rh;
    xl[o0] = rl;
    xh[o1] = ih;
    xl[o1] = il;
    xh[o2] = -rh;
    xl[o2] = -rl;
  }
#pragma unroll
  for (int j = 0; j < TC_PER_WARP - 4; ++j) {
    if (g0 + 2 * j >= ngw) continue;
    float rh, rl, ih, il;
    split(raw[(2 * (4 + j)) * TC_PROD + tid], rh, rl);
    split(raw[(2 * (4 + j) + 1) * TC_PROD + tid], ih, il);
    const uint32_t o = base + (uint32_t)(2 * j * TC_GRP / 4);
    w[o] = rh;
    w[o + TC_WTILE / 4] = rl;
    w[o + 2 * TC_WTILE / 4] = ih;
    w[o + 3 * TC_WTILE / 4] = il;
  }
}

// What the epilogue of a tile needs, written by the MMA-issuing thread into the accumulator's
// record before it releases the accumulator's "full" barrier.
struct EpiRec {
  float* c;          // C element (m0, 0) of the real plane
  int64_t plane, ld;
  int32_t rows, n;
  float alpha, beta;
  int32_t pad[2];
};
static_assert(sizeof(EpiRec) == 48, "epilogue record size");

// C rows of a tile from TMEM accumulator acc (D columns = rows of the tile, lanes = right-hand
// sides and planes); ew = epilogue warp 0..3 reads TMEM lanes 32 ew .. 32 ew + 31.  Groups of
// 32 rows: the group's C values (beta != 0) are requested before its TMEM load, so that one
// memory latency is paid per group.
__device__ __forceinline__ void epilogue(const EpiRec& er, uint32_t acc, int ew, int lane) {
  const int rows = er.rows;
  const int q = ew * 32 + lane;               // TMEM lane = row of D
  const int col = q & 63;                     // right-hand side
  const bool act = col < er.n;
  const float alpha = er.alpha, beta = er.beta;
  const int64_t ld = er.ld;
  float* const C = er.c + (q >= 64 ? er.plane : 0) + col;
  const uint32_t lane_base = (uint32_t)(ew * 32) << 16;
#pragma unroll 1
  for (int c0 = 0; c0 < rows; c0 += 32) {
    float old[32];
    if (beta != 0.f) {
#pragma unroll
      for (int e = 0; e < 32; ++e) old[e] = (act && c0 + e < rows) ? C[(int64_t)(c0 + e) * ld] : 0.f;
    }
    uint32_t v[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(acc + lane_base + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (act) {
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        if (c0 + e < rows) {
          float val = alpha * __uint_as_float(v[e]);
          if (beta != 0.f) val += beta * old[e];
          C[(int64_t)(c0 + e) * ld] = val;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_nrhs_tc(const GemmDesc<float>* __restrict__ descs,
                                                                 const GemmTile* __restrict__ tiles, int ntiles,
                                                                 int32_t* status, long long spins) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if ((int)blockIdx.x >= ntiles) return;
  const uint32_t sbase = (smem_u32(smem) + 1023u) & ~1023u;
  unsigned char* sgen = smem + (sbase - smem_u32(smem));
  const uint32_t raw0 = sbase + TC_OFF_RAW;
  const float* rawg = reinterpret_cast<const float*>(sgen + TC_OFF_RAW);
  const GemmDesc<float>* sd = reinterpret_cast<const GemmDesc<float>*>(sgen + TC_OFF_DESC);
  const GemmTile* st = reinterpret_cast<const GemmTile*>(sgen + TC_OFF_TILE);
  const uint32_t sd_u = sbase + TC_OFF_DESC, st_u = sbase + TC_OFF_TILE;
  EpiRec* erec = reinterpret_cast<EpiRec*>(sgen + TC_OFF_EREC);
  const uint32_t bar0 = sbase + TC_OFF_BAR;                 // slot barriers
  const uint32_t bar_full = bar0 + 8 * TC_SLOTS;            // accumulator a complete
  const uint32_t bar_empty = bar_full + 8 * TC_NACC;        // accumulator a read (4 epilogue warps)
  const uint32_t bar_spare = bar_empty + 8 * TC_NACC;       // nothing arrives here
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sgen + TC_OFF_MISC);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sgen + TC_OFF_MISC + 4);
  if (tid == 0) {
    for (int s = 0; s < TC_SLOTS; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar0 + 8 * s), "r"(1));
    for (int a = 0; a < TC_NACC; ++a) {
      // full: the MMAs' commit and thread 0's arrive after writing the epilogue record
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar_full + 8 * a), "r"(2));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar_empty + 8 * a), "r"(TC_EPI / 32));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar_spare), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    *abort_flag = 0;
  }
  // the first tiles' records and descriptors, synchronously
  for (int x = tid; x < TC_TAHEAD; x += TC_THREADS) {
    const int t = (int)blockIdx.x + x * (int)gridDim.x;
    if (t < ntiles) const_cast<GemmTile*>(st)[x] = tiles[t];
  }
  __syncthreads();
  for (int x = tid; x < TC_DAHEAD * (TC_DESC_BYTES / 16); x += TC_THREADS) {
    const int o = x / (TC_DESC_BYTES / 16), part = x % (TC_DESC_BYTES / 16);
    const int t = (int)blockIdx.x + o * (int)gridDim.x;
    if (t < ntiles)
      reinterpret_cast<int4*>(sgen + TC_OFF_DESC + o * TC_DESC_BYTES)[part] =
          reinterpret_cast<const int4*>(descs + st[o].desc)[part];
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
    ok = __syncthreads_and(mbar_wait(bar_spare, 0u, spins) ? 1 : 0) != 0;
  long long g = 0;      // chunks taken by this CTA (producers)
  long long gi = 0;     // chunks whose MMAs the MMA warp issued (g - 1 at most after an expired wait)
  if (tid < TC_PROD) {
    // ---------------- producers ----------------
    Cursor cur;
    cur.t = ok ? (int)blockIdx.x : ntiles;   // after an expired test wait the CTA issues no work
    Cursor cp = cur;
    // copies run TC_NRAW - 1 chunks ahead of use: chunk g + TC_NRAW - 1 is requested while g is used
    for (int s = 0; s < TC_NRAW - 1; ++s) {
      if (cp.t < ntiles) {
        if (cp.c == 0 && warp == 1) fetch_records(cp.i, ntiles, descs, tiles, sd_u, st_u, st, lane);
        copy_chunk(raw0 + s * TC_RAW, sd[cp.i % TC_DRING], st[cp.i % TC_TRING], cp.c, descs, warp, lane, tid);
        advance(cp, sd);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
#pragma unroll 1
    while (cur.t < ntiles) {
      const GemmDesc<float>& d = sd[cur.i % TC_DRING];
      const GemmTile tl = st[cur.i % TC_TRING];
      const int nk = tile_chunks(d);
      const int rows = min(TC_ROWS, d.m - tl.tm * TC_ROWS);
      const int nt = (rows + 15) & ~15;
      const int slot = (int)(g % TC_SLOTS);
      unsigned char* sp = sgen + slot * TC_SLOT;
      const bool last = cur.c + 1 == nk;
      // request chunk g + TC_NRAW - 1 (and records), then wait for this thread's copies of chunk g
      if (cp.t < ntiles) {
        if (cp.c == 0 && warp == 1) fetch_records(cp.i, ntiles, descs, tiles, sd_u, st_u, st, lane);
        copy_chunk(raw0 + (int)((g + TC_NRAW - 1) % TC_NRAW) * TC_RAW, sd[cp.i % TC_DRING], st[cp.i % TC_TRING], cp.c,
                   descs, warp, lane, tid);
        advance(cp, sd);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group %0;\n" ::"n"(TC_NRAW - 1) : "memory");
      // the slot is free: the MMA warp passed the last barrier after chunk g - 2's MMAs completed
      if (ok) store_chunk(rawg + (size_t)(g % TC_NRAW) * (TC_RAW / 4), sp, nt / 8, warp, lane, tid);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      if (chunk_sync_or(!ok || *abort_flag)) {
        ok = false;
        break;
      }
      ++g;
      if (last) {
        cur.c = 0;
        cur.t += gridDim.x;
        ++cur.i;
      } else {
        ++cur.c;
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");   // no copy may land after the CTA is gone
    if (!ok) *abort_flag = 1;
  } else if (warp == TC_MMA_WARP) {
    // ---------------- MMA warp: the producers' cursor, one chunk behind them ----------------
    Cursor cur;
    cur.t = ok ? (int)blockIdx.x : ntiles;
#pragma unroll 1
    while (cur.t < ntiles) {
      const GemmDesc<float>& d = sd[cur.i % TC_DRING];
      const GemmTile tl = st[cur.i % TC_TRING];
      const int nk = tile_chunks(d);
      const int rows = min(TC_ROWS, d.m - tl.tm * TC_ROWS);
      const int nt = (rows + 15) & ~15;
      const int slot = (int)(g % TC_SLOTS);
      const uint32_t sa = sbase + slot * TC_SLOT;
      const bool last = cur.c + 1 == nk;
      // chunk g - 1's MMAs complete before the barrier, after which the producers refill its slot
      if (lane == 0 && ok && g >= 1)
        ok = mbar_wait_or_abort(bar0 + 8 * (int)((g - 1) % TC_SLOTS), (uint32_t)(((g - 1) / TC_SLOTS) & 1), spins,
                                abort_flag);
      __syncwarp();
      if (chunk_sync_or(!ok || *abort_flag)) {   // chunk g is in its slot
        ok = false;
        break;
      }
      const int a = cur.i % TC_NACC;
      const uint32_t acc_tm = tmem + (uint32_t)(a * 128);
      if (lane == 0) {
        // a tile's first chunk reuses the accumulator of tile i - TC_NACC: wait until it has been read
        if (cur.c == 0 && cur.i >= TC_NACC)
          ok = mbar_wait_or_abort(bar_empty + 8 * a, (uint32_t)(((cur.i / TC_NACC) - 1) & 1), spins, abort_flag);
        if (ok) {
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
          const uint32_t id_p = idesc(nt, 0), id_n = idesc(nt, 1);
          const uint32_t xh = sa, xl = sa + TC_XTILE;
          const uint32_t x2 = 8 * TC_GRP;   // rows 64.. of the X stack
          const uint32_t wrh = sa + 2 * TC_XTILE, wrl = wrh + TC_WTILE, wih = wrh + 2 * TC_WTILE,
                         wil = wrh + 3 * TC_WTILE;
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
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           bar0 + 8 * slot)
                       : "memory");
          if (last) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             bar_full + 8 * a)
                         : "memory");
            EpiRec& er = erec[a];
            er.c = d.C.re + (int64_t)tl.tm * TC_ROWS * d.C.ld;
            er.plane = d.C.plane;
            er.ld = d.C.ld;
            er.rows = rows;
            er.n = d.n;
            er.alpha = d.alpha;
            er.beta = d.beta;
            mbar_arrive(bar_full + 8 * a);   // release: the record is visible to the epilogue warps
          }
          gi = g + 1;
        } else {
          *abort_flag = 1;
        }
      }
      __syncwarp();   // the warp meets the next aligned barrier converged
      ++g;
      if (last) {
        cur.c = 0;
        cur.t += gridDim.x;
        ++cur.i;
      } else {
        ++cur.c;
      }
    }
    if (!ok) *abort_flag = 1;
  } else {
    // ---------------- epilogue warps ----------------
    const int ew = warp - TC_WARPS;   // TMEM lanes 32 ew .. 32 ew + 31 (warp % 4 == ew)
    int j = 0;
#pragma unroll 1
    for (int t = (int)blockIdx.x; ok && t < ntiles; t += gridDim.x, ++j) {
      const int a = j % TC_NACC;
      const bool got = mbar_wait_or_abort(bar_full + 8 * a, (uint32_t)((j / TC_NACC) & 1), spins, abort_flag);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      epilogue(erec[a], tmem + (uint32_t)(a * 128), ew, lane);
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_empty + 8 * a);
    }
  }
  __syncthreads();
  // drain: every MMA this CTA issued has completed before TMEM is released (with the default
  // limit even after an expired wait, so that no MMA can still write the columns being freed)
  if (warp == TC_MMA_WARP && lane == 0 && gi > 0) {
    const int slot = (int)((gi - 1) % TC_SLOTS);
    if (!mbar_wait(bar0 + 8 * slot, (uint32_t)(((gi - 1) / TC_SLOTS) & 1), kDefaultWaitLimit)) ok = false;
  }
  if (*abort_flag) ok = false;
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
  const int grid = ntiles < sms ? ntiles : sms;   // one CTA per SM
  count_launches(1);
  k_gemm_nrhs_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(d_desc, d_tiles, ntiles, status, wait_limit());
}

}  // namespace mf
