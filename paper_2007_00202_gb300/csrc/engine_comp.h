// Compressed fronts of the multifrontal factorization (Alg. 5, lines 8-12) on the GPU:
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
      : an_(an), A_(A), st_(st), cx(st, persist, scratch) {}

  // Factor compressed front fid.  fr: dense-front descriptors (children's dense C blocks live there).
  void factor_front(int fid, const std::vector<FrontDev<T>>& fr, const BFParams& P, uint64_t seed);
  // Expand C of a compressed front into the dense buffer of its (dense) parent's extend-add.
  void densify_C(int fid, const FrontDev<T>& f);
  // Solve steps on X (N x k, planar row-major, new numbering) for all compressed fronts of one
  // tree level at once (they touch disjoint separator rows; the update rows they write are
  // combined by the scatter-add of the forward step)
  void forward(const std::vector<int>& fids, Blk<T>& X);
  void backward(const std::vector<int>& fids, Blk<T>& X);

  const Analysis& an_;
  const DeviceMatrix& A_;
  cudaStream_t st_;
  BFContext<T> cx;
  std::map<int, std::unique_ptr<CompFront<T>>> fronts;
};

}  // namespace mf
