// Device butterfly and HOD-BF matrices (Sec. 3-4) and their algorithms on the GPU:
// apply / transpose apply, extraction of sub-block lists (Alg. 3), construction
// from entry extraction (Alg. 2) and from products (Sec. 3.2), HOD-BF
// construction, extraction and inversion (Alg. 4 with BF_SMW).
//
// Control flow runs on the host (index sets, ranks and skeletons are host
// data, exactly as the oracle keeps them); every numerical step is a batched
// device launch: one GEMM launch per butterfly level for all blocks of all
// butterflies involved, one batched ID launch per construction level.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <functional>
#include <memory>
#include <chrono>
#include <string>
#include <map>
#include <vector>

#include "analysis.h"
#include "bf_kernels.h"
#include "engine.h"

namespace mf {

using Tree = std::vector<std::vector<Range>>;   // levels of index ranges

// Bump allocator over one device allocation; mark/release for scratch phases.  An arena can
// instead forward every request to a shared parent arena (share()): several construction
// contexts then allocate their persistent blocks from one allocation, under the parent's lock.
class Arena {
 public:
  void init(size_t bytes) {
    mem_.alloc(bytes);
    off_ = 0;
  }
  void share(Arena* parent) { parent_ = parent; }
  bool ready() const { return parent_ ? parent_->ready() : mem_.p != nullptr; }
  void* take(size_t bytes) {
    if (parent_) return parent_->take(bytes);
    std::lock_guard<std::mutex> lk(mu_);
    size_t o = (off_ + 255) & ~size_t(255);
    if (o + bytes > mem_.bytes)
      throw CudaError("device arena exhausted (cudaMalloc: out of memory): need " + std::to_string(o + bytes) +
                      " of " + std::to_string(mem_.bytes) + " bytes");
    off_ = o + bytes;
    peak_ = std::max(peak_, off_);
    return static_cast<char*>(mem_.p) + o;
  }
  template <typename T>
  T* takeT(size_t n) { return static_cast<T*>(take(n * sizeof(T))); }
  // mark / release are meant for an arena used by one thread (the scratch arenas); on a shared
  // arena they act on the parent
  size_t mark() const { return parent_ ? parent_->mark() : off_; }
  void release(size_t m) {
    if (parent_) {
      parent_->release(m);
      return;
    }
    std::lock_guard<std::mutex> lk(mu_);
    off_ = m;
  }
  size_t used() const { return parent_ ? 0 : off_; }
  size_t peak() const { return parent_ ? 0 : peak_; }          // a shared arena counts in its parent
  size_t capacity() const { return parent_ ? 0 : mem_.bytes; }
  char* base() const { return parent_ ? parent_->base() : static_cast<char*>(mem_.p); }

 private:
  DevMem mem_;
  size_t off_ = 0, peak_ = 0;
  Arena* parent_ = nullptr;
  std::mutex mu_;
};

// A planar complex block in device memory: rows x cols, row-major, leading dim ld.
template <typename T>
struct Blk {
  T* p = nullptr;
  int64_t plane = 0;
  int32_t rows = 0, cols = 0;
  int64_t ld = 0;
  PMat<T> pm() const { return PMat<T>{p, plane, ld}; }
  Blk sub(int r0, int c0, int nr, int nc) const {
    Blk b = *this;
    b.p = p + (int64_t)r0 * ld + c0;
    b.rows = nr;
    b.cols = nc;
    return b;
  }
};

template <typename T>
Blk<T> new_blk(Arena& a, int rows, int cols) {
  Blk<T> b;
  b.rows = rows;
  b.cols = cols;
  b.ld = std::max(1, (cols + 3) & ~3);
  b.plane = (int64_t)std::max(rows, 1) * b.ld;
  b.p = a.takeT<T>(2 * (size_t)b.plane);
  return b;
}

using IdxVec = std::vector<int32_t>;

// Device butterfly (hybrid form, centre at l_c = floor(L/2)).
template <typename T>
struct DBF {
  int m = 0, n = 0, L = 0, lc = 0;
  Tree rt, ct;
  // index of pair (i, j) at level l: i * 2^(L-l) + j
  std::vector<std::vector<Blk<T>>> U;     // l in [lc, L]   (U at L, R below)
  std::vector<std::vector<IdxVec>> Osk;
  std::vector<std::vector<Blk<T>>> V;     // l in [0, lc]   (V at 0, W above)
  std::vector<std::vector<IdxVec>> Ssk;
  std::vector<Blk<T>> B;                  // pairs at lc
  void init(int m_, int n_, const Tree& r, const Tree& c, int L_) {
    m = m_; n = n_; L = L_; lc = L_ / 2;
    rt.assign(r.begin(), r.begin() + L_ + 1);
    ct.assign(c.begin(), c.begin() + L_ + 1);
    U.assign(L + 1, {}); Osk.assign(L + 1, {});
    V.assign(L + 1, {}); Ssk.assign(L + 1, {});
    for (int l = 0; l <= L; ++l) {
      size_t np = (size_t)1 << L;
      if (l >= lc) { U[l].resize(np); Osk[l].resize(np); }
      if (l <= lc) { V[l].resize(np); Ssk[l].resize(np); }
    }
    B.resize((size_t)1 << L);
  }
  int pidx(int l, int i, int j) const { return i * (1 << (L - l)) + j; }
  int rr(int l, int i, int j) const { return (int)Osk[l][pidx(l, i, j)].size(); }
  int rc(int l, int i, int j) const { return (int)Ssk[l][pidx(l, i, j)].size(); }
  int max_rank() const;
  double storage() const;   // complex entries
};

// HOD-BF matrix over a uniform-depth cluster tree.
template <typename T>
struct DHODBF {
  int n = 0, LH = 0;
  Tree tree;
  std::vector<Blk<T>> D;                   // leaves
  std::vector<std::vector<std::unique_ptr<DBF<T>>>> off;   // off[l][i], l = 1..LH: K(node i, sibling)
  int max_rank() const;
  double storage() const;
};

// HOD-BF inverse in the product form of Alg. 4:
// D^-1 = M_root diag(M_level1) ... diag(M_level(LH-1)) diag(D_leaf^-1), M = I + K.
template <typename T>
struct DHODBFInv {
  int n = 0, LH = 0;
  Tree tree;
  std::vector<Blk<T>> Dinv;
  std::vector<std::vector<std::unique_ptr<DBF<T>>>> M;    // M[l][i], l = 0..LH-1
  double storage() const;
};

// A black-box operator on device vectors: Y = K X (or K^T X); X is cols x k,
// Y rows x k, both row-major planar (ld = k, plane = rows * k).
template <typename T>
struct DOp {
  int rows = 0, cols = 0;
  std::function<void(const Blk<T>& X, Blk<T>& Y, bool transpose)> apply;
};

// Extraction callback: fills dst blocks (allocated by the caller, X.size() x Y.size()).
template <typename T>
using DExtract = std::function<void(const std::vector<std::pair<IdxVec, IdxVec>>& lst, std::vector<Blk<T>>& dst)>;

// One butterfly construction problem of a batch (Alg. 2 in lockstep).
template <typename T>
struct BFProblem {
  int m = 0, n = 0, L = 0;
  int64_t row_off = 0, col_off = 0;   // shift of local indices into the extractor's index space
  Tree rt, ct;
  std::vector<IdxVec> nn_r, nn_c;     // neighbour lists in local indices
  std::unique_ptr<DBF<T>> out;
};

// One HOD-BF construction problem: square block of size n at offset off of the extractor's index space.
template <typename T>
struct HProblem {
  int n = 0;
  int64_t off = 0;
  Tree tree;
  const std::vector<IdxVec>* nn = nullptr;   // neighbours in local indices (owned by the caller)
  std::unique_ptr<DHODBF<T>> out;
};

// Batched black-box operator: Y[q] = K_q X[q] (or K_q^T X[q]) for every problem q of a batch.
template <typename T>
using DOpB = std::function<void(const std::vector<Blk<T>>& X, std::vector<Blk<T>>& Y, bool transpose)>;

// One randomized construction problem of a batch (all problems of a batch share L).
template <typename T>
struct RMProblem {
  int m = 0, n = 0;
  Tree rt, ct;
  uint32_t key = 0;
  std::unique_ptr<DBF<T>> out;
};

// One BF_SMW assembly problem: quadrants of K (K11, K22i may be null) on tree tr.
template <typename T>
struct SmwItem {
  int n = 0;
  Tree tr;
  const DBF<T>* K11 = nullptr;
  const DBF<T>* K12 = nullptr;
  const DBF<T>* K21 = nullptr;
  const DBF<T>* K22i = nullptr;
  uint32_t key = 0;
  std::unique_ptr<DBF<T>> out;
};

struct BFParams {
  double tol = 1e-4;
  int max_rank = 0;
  int alpha = 2, knn = 8;
  int p = 8;            // oversampling of the randomized construction
  int q_start = 64;     // sketch width without a rank cap
};

// Everything the butterfly algorithms need: stream, arenas, counters.
template <typename T>
class BFContext {
 public:
  BFContext(cudaStream_t st, size_t persist_bytes, size_t scratch_bytes);
  // a context whose persistent blocks come from another context's persistent arena
  BFContext(cudaStream_t st, Arena* shared_persist, size_t scratch_bytes);
  ~BFContext();
  cudaStream_t st;
  cudaStream_t side[2] = {nullptr, nullptr};            // forked streams of row_ids (created on first use)
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  char* ring = nullptr;             // pinned host staging ring
  char* ring_dev = nullptr;         // the ring's device-mapped address (kernels read it in place)
  DevMem dring;                     // a device mirror of the ring, where mapping is not available
  size_t ring_cap = 0, ring_off = 0, pend_begin = 0;
  bool pend = false;
  int64_t n_copies = 0;             // host -> device copies issued
  char* cap_host = nullptr;         // capture blob (pinned host) and its device twin
  char* cap_dev = nullptr;
  size_t cap_cap = 0, cap_off = 0;
  bool cap_bad = false;
  double t_wait = 0;                // seconds the host spent waiting for the stream
  LaunchProfiler* prof = nullptr;   // event timing of the narrow GEMM launches (when on)
  // host seconds spent inside the main routines (inclusive; read by the MF_TRACE=1 phase trace)
  enum { H_GEMM, H_ROWID, H_APPLY, H_EXTRACT, H_PROXY, H_RMV, H_BLK2, H_SKETCH, H_UPLOAD, H_HEXTRACT, H_EXT, H_N };
  double t_host[H_N] = {};
  struct HostTimer {
    double* acc;
    std::chrono::steady_clock::time_point t0;
    explicit HostTimer(double* a) : acc(a), t0(std::chrono::steady_clock::now()) {}
    ~HostTimer() { *acc += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  };
  Arena persist, scratch;
  DevMem status;
  double flops = 0;
  double bytes = 0;   // algorithmic bytes of the products issued (factor blocks, inputs and outputs)
  int max_rank_seen = 0;
  int64_t n_id = 0;

  // ---- primitives
  // Asynchronous host -> device copy of small host data through a pinned staging ring (the
  // host data may be reused as soon as the call returns).
  void h2d(void* dst, const void* src, size_t bytes);
  // Small host arrays read by this context's kernels (index lists) are staged in the ring:
  // upload() copies the bytes there and returns their device address in the mirror; the
  // staged bytes go to the device in one cudaMemcpyAsync per run, issued by flush().  h2d()
  // flushes first, and every launch is preceded by the h2d of its job table, so a kernel
  // always finds the index lists its jobs point to.
  const void* upload(const void* src, size_t bytes);
  void flush();
  // upload + flush: a job table that the next launch reads
  template <typename U>
  const U* stage(const U* src, size_t n) {
    const U* d = static_cast<const U*>(upload(src, n * sizeof(U)));
    flush();
    return d;
  }
  // ---- CUDA-graph capture of a fixed launch sequence (the compressed solve)
  // count_begin/count_end measure the staged bytes of one eager run of the sequence;
  // capture_begin redirects staging into a persistent pinned blob (host) whose device
  // twin the captured kernels read, and capture_end copies the blob to the device
  // once.  A stream synchronize or an overflow while capturing marks the capture bad.
  void count_begin() { cap_mode = 1; cap_off = 0; }
  size_t count_end() { cap_mode = 0; return cap_off; }
  void capture_begin(char* host_blob, char* dev_blob, size_t cap) {
    cap_mode = 2; cap_host = host_blob; cap_dev = dev_blob; cap_cap = cap; cap_off = 0; cap_bad = false;
  }
  bool capture_end();               // after cudaStreamEndCapture; false if the capture is unusable
  int cap_mode = 0;                 // 0 eager, 1 counting, 2 capturing
  void sync();                      // stream synchronize, timed into t_wait
  void gemm(std::vector<GemmDesc<T>>& descs);             // one launch for all descs
  // consecutive dependent launches (stage s reads what stage s - 1 wrote): one upload of every
  // stage's descriptors and tiles when all run on the tensor-core kernel, else gemm() per stage
  void gemm_stages(std::map<int, std::vector<GemmDesc<T>>>& stages);
  void zero(Blk<T>& b);                                   // b: a whole block from new_blk
  // row IDs of the given matrices (device); results on host (ranks, skeletons) and U in persist
  // centre blocks by least squares, one launch for all jobs (work from scratch when shared memory is short)
  void run_lstsq(std::vector<LstsqJob<T>>& lj);
  void row_ids(const std::vector<Blk<T>>& Ms, double tol, int max_rank, std::vector<IdxVec>& sk,
               std::vector<Blk<T>>& Us);
  // ---- butterfly algorithms
  void apply(const std::vector<const DBF<T>*>& bfs, const std::vector<Blk<T>>& X, std::vector<Blk<T>>& Y,
             bool transpose, bool accumulate);
  void extract_bf(const DBF<T>& bf, const std::vector<std::pair<IdxVec, IdxVec>>& lst, std::vector<Blk<T>>& dst,
                  T sign);
  // several butterflies at once, stage-merged; dst blocks receive += K(X, Y)
  void extract_multi(const std::vector<const DBF<T>*>& bfs,
                     const std::vector<const std::vector<std::pair<IdxVec, IdxVec>>*>& lsts,
                     const std::vector<std::vector<Blk<T>>*>& dsts);
  void entry_eval_batch(const DExtract<T>& ext, std::vector<BFProblem<T>>& probs, const BFParams& P);
  void hodbf_entry_eval_batch(const DExtract<T>& ext, std::vector<HProblem<T>>& probs, const BFParams& P);
  std::unique_ptr<DBF<T>> entry_eval(const DExtract<T>& ext, int m, int n, const Tree& rt, const Tree& ct, int L,
                                      const std::vector<IdxVec>& nn_r, const std::vector<IdxVec>& nn_c,
                                      const BFParams& P);
  std::unique_ptr<DBF<T>> random_matvec(const DOp<T>& op, const Tree& rt, const Tree& ct, int L, const BFParams& P,
                                         uint32_t key);
  void right_transform(const DBF<T>& bf, const Blk<T>& X, std::vector<Blk<T>>& xs);
  std::unique_ptr<DBF<T>> split_child(const DBF<T>& bf, int a, int b);
  // ---- HOD-BF
  std::unique_ptr<DHODBF<T>> hodbf_entry_eval(const DExtract<T>& ext, int n, const Tree& tree,
                                               const std::vector<IdxVec>& nn, const BFParams& P);
  void hodbf_apply(const DHODBF<T>& H, const Blk<T>& X, Blk<T>& Y, bool transpose);
  void hodbf_extract(const DHODBF<T>& H, const std::vector<std::pair<IdxVec, IdxVec>>& lst, std::vector<Blk<T>>& dst,
                     T sign);
  std::unique_ptr<DHODBFInv<T>> hodbf_invert(const DHODBF<T>& H, const BFParams& P, uint32_t key);
  void inv_apply(const DHODBFInv<T>& Hi, const Blk<T>& X, Blk<T>& Y, bool transpose, int l0 = 0, int i0 = 0);
  // Y_q = H_q^-1 X_q (or H_q^-T X_q) for several full inverses at once, in lockstep
  void inv_apply_multi(const std::vector<const DHODBFInv<T>*>& His, const std::vector<Blk<T>>& X,
                       std::vector<Blk<T>>& Y, bool transpose);
  std::unique_ptr<DBF<T>> bf_smw(const DBF<T>& K, const BFParams& P, uint32_t key);
  std::unique_ptr<DBF<T>> smw_assemble(int n, const Tree& tr, int L, const DBF<T>* K11, const DBF<T>& K12,
                                       const DBF<T>& K21, const DBF<T>* K22i, const BFParams& P, uint32_t key);
  void check_status();
  // ---- batched forms (all problems of one call in lockstep)
  Blk<T> make_sketch(int rows, const std::vector<Range>& groups, int q, int level, int side, uint32_t key,
                     std::vector<std::pair<int, int>>& cols);
  // the sketches of several levels side by side in one block: level k's columns start at base[k],
  // its groups' column ranges (relative to base[k]) in cols[k]; one launch
  Blk<T> make_sketch_levels(int rows, const std::vector<std::pair<const std::vector<Range>*, int>>& lv, int q,
                            int side, uint32_t key, std::vector<std::vector<std::pair<int, int>>>& cols,
                            std::vector<int>& base);
  void random_matvec_batch(const DOpB<T>& op, std::vector<RMProblem<T>>& probs, int L, const BFParams& P);
  void inv_apply_b(const DHODBFInv<T>& Hi, int l0, const std::vector<int>& i0s, const std::vector<Blk<T>>& X,
                   std::vector<Blk<T>>& Y, bool transpose);
  std::vector<std::unique_ptr<DBF<T>>> bf_smw_batch(const std::vector<const DBF<T>*>& Ks,
                                                    const std::vector<uint32_t>& keys, const BFParams& P);
  void smw_assemble_batch(std::vector<SmwItem<T>>& items, int L, const BFParams& P);
  std::vector<Blk<T>> copy_b(const std::vector<Blk<T>>& x);
  void axpy_b(const std::vector<Blk<T>>& x, std::vector<Blk<T>>& y, T alpha);
};

}  // namespace mf
