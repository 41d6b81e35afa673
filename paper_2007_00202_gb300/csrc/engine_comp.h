// Compressed fronts of the multifrontal factorization (the large-front branch of Alg. 5) on the GPU:
//   F11   <- HODBF_entry_eval(A(Is,Is) (+) C_nu1 (+) C_nu2)
//   F11^-1<- HODBF_invert(F11)                                 (Alg. 4)
//   F12   <- BF_entry_eval(A(Is,Iu) (+) C_nu1 (+) C_nu2)        (Alg. 2)
//   F21   <- BF_entry_eval(A(Iu,Is) (+) C_nu1 (+) C_nu2)
//   S     <- BF_random_matvec(F21 F11^-1 F12)                  (Sec. 3.2)
//   C_tau <- HODBF_entry_eval(C_nu1 (+) C_nu2 - S)
// Entries come from A, dense children (gathers) and compressed children
// (extract_HODBF), split per source as in Sec. 5 step 1.  Solve (block LU):
// forward w = F11^-1 b_s, b_u -= F21 w; backward x_s = w - F11^-1 F12 x_u.
#pragma once
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "bf_engine.h"

namespace mf {

template <typename T>
struct CompFront {
  int fid = -1;
  int s = 0, u = 0;
  int64_t sep_begin = 0;
  std::unique_ptr<DHODBF<T>> F11;
  std::unique_ptr<DHODBFInv<T>> F11inv;
  std::unique_ptr<DBF<T>> F12, F21;
  std::unique_ptr<DHODBF<T>> C;
  IdxVec upd32;
  DevMem d_upd32, d_iota;
  int max_rank = 0;
  double seconds = 0;
};

template <typename T>
class CompressedPart {
 public:
  CompressedPart(const Analysis& an, const DeviceMatrix& A, cudaStream_t st, size_t persist, size_t scratch)
      : an_(an), A_(A), st_(st), cx(st, persist, scratch), persist_bytes_(persist), scratch_bytes_(scratch) {}
  ~CompressedPart() {
    extra_.clear();
    for (auto s : extra_st_)
      if (s) cudaStreamDestroy(s);
  }
  // the most construction contexts (host threads and streams) that build the fronts of one level
  static constexpr int kMaxContexts = 8;

  // Factor compressed front fid with execution context w (0: the engine's stream and arenas,
  // 1: a second context on its own stream, so that two fronts of one tree level can be built
  // by two host threads at once).  fr: dense-front descriptors (children's dense C blocks).
  // w: the context that builds the front; helper >= 0: a second context that builds F12 and F21
  // at the same time
  void factor_front(int fid, const std::vector<FrontDev<T>>& fr, const BFParams& P, uint64_t seed, int w = 0,
                    int helper = -1);
  // Expand C of a compressed front into the dense buffer of its (dense) parent's extend-add.
  void densify_C(int fid, const FrontDev<T>& f, int w = 0);
  // execution contexts 1 .. n-1 (created on first use, each with its own stream and scratch arena;
  // their persistent blocks come from context 0's persistent arena)
  void ensure_contexts(int n);
  int contexts() const { return 1 + (int)extra_.size(); }
  BFContext<T>& ctx(int w) { return w == 0 ? cx : *extra_[w - 1]; }
  cudaStream_t stream(int w) const { return w == 0 ? st_ : extra_st_[w - 1]; }
  // Solve steps on X (N x k, planar row-major, new numbering) for all compressed fronts of one
  // tree level at once (they touch disjoint separator rows; the update rows they write are
  // combined by the scatter-add of the forward step)
  void forward(const std::vector<int>& fids, Blk<T>& X);
  void backward(const std::vector<int>& fids, Blk<T>& X);

  // Neighbour lists of a compressed front in front positions (the proxy candidates of Sec. 5.2):
  // nn11 (I^s -> I^s), nn12 (I^s -> I^u, local), nn21 (I^u -> I^s), nn22 (I^u -> I^u, local).
  // They depend on the graph and the trees only, so they are computed once per analysis.
  struct Neigh {
    std::vector<IdxVec> nn11, nn12, nn21, nn22;
  };
  // computes the lists of every compressed front (several host threads); factor_front computes a
  // missing entry itself
  void prepare_neighbours(int knn);
  const Neigh& neighbours(int fid, int knn);

  const Analysis& an_;
  const DeviceMatrix& A_;
  cudaStream_t st_;
  BFContext<T> cx;
  std::vector<std::unique_ptr<BFContext<T>>> extra_;
  std::vector<cudaStream_t> extra_st_;
  size_t persist_bytes_, scratch_bytes_;
  std::mutex fronts_mu_;   // guards fronts while two contexts build fronts of one level
  std::map<int, std::unique_ptr<CompFront<T>>> fronts;
  std::mutex neigh_mu_;
  std::map<int, std::unique_ptr<Neigh>> neigh_;   // per front, for neigh_knn_
  int neigh_knn_ = -1;
};

}  // namespace mf
