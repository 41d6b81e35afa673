// Host-side symbolic analysis of the multifrontal method (Sec. 2, Sec. 5.1, Sec. 5.2).
// Written independently of the oracle from the same rules; the two must agree bit for bit.
#pragma once
#include <cstdint>
#include <vector>

namespace mf {

struct Range { int64_t a, b; };

struct FrontInfo {
  int64_t id = 0;
  int64_t parent = -1;
  std::vector<int64_t> children;
  int64_t sep_begin = 0, sep_end = 0;   // I^s = [sep_begin, sep_end) in the new numbering
  int64_t sub_begin = 0;                // first new index of the subtree
  std::vector<int64_t> upd;             // I^u, sorted new indices
  int32_t level = 0;                    // depth in the assembly tree (root 0)
  bool compressed = false;
  std::vector<std::vector<Range>> th_tree;   // HOD-BF cluster tree of F11 (levels of ranges over [0,s))
  std::vector<std::vector<Range>> f22_tree;  // cluster tree of F22 (levels of ranges over [0,u))
  int64_t s() const { return sep_end - sep_begin; }
  int64_t u() const { return (int64_t)upd.size(); }
};

struct Analysis {
  int64_t n = 0;
  std::vector<int64_t> perm, iperm;     // perm[new] = old
  std::vector<FrontInfo> fronts;        // post-order
  std::vector<int64_t> prow;            // permuted pattern (CSR, sorted)
  std::vector<int64_t> pcol;
  int32_t leaf_size = 64, nmin_sep = 1024, hodbf_leaf = 64;
};

enum { LATTICE_NODE = 0, LATTICE_EDGE = 1 };

// Throws std::runtime_error on invalid input.
// ordering: ORDER_AUTO (planar with coords, graph without), ORDER_HYBRID (planar separators while
// they are compressed, graph nested dissection of every box whose planar separator is smaller
// than nmin_sep), ORDER_GRAPH (graph nested dissection even with coords)
enum { ORDER_AUTO = 0, ORDER_HYBRID = 1, ORDER_GRAPH = 2 };
// parallel_levels: the planar rule cuts the boxes of the top parallel_levels levels along the root's
// axis (while they extend 3 or more units along it), so that those separators are parallel planes
void analyze(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* coords, int lattice,
             int leaf_size, int nmin_sep, int hodbf_leaf, Analysis& out, int ordering = ORDER_AUTO,
             int parallel_levels = 0);

std::vector<std::vector<Range>> cluster_tree_balanced(int64_t npts, int64_t leaf);

// Breadth-first search nearest neighbours (Sec. 5.2).
void bfs_nearest(const Analysis& an, int64_t start, const std::vector<uint8_t>& allowed,
                 const std::vector<uint8_t>& target, int knn, std::vector<int64_t>& out,
                 std::vector<int64_t>& stamp, int64_t& stamp_val);

struct FrontNeighbours {
  // CSR-like: for each vertex of the set (in order), up to knn neighbours (new indices)
  std::vector<int64_t> nn11_ptr, nn11;  // rows I^s (in order)
  std::vector<int64_t> nn22_ptr, nn22;  // rows I^u (in order)
  std::vector<int64_t> nn12_ptr, nn12;  // rows I^s -> vertices of I^u
  std::vector<int64_t> nn21_ptr, nn21;  // rows I^u -> vertices of I^s
};
void front_neighbours(const Analysis& an, const FrontInfo& f, int knn, FrontNeighbours& out);

}  // namespace mf
