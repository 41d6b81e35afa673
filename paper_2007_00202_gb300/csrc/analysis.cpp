// Host-side symbolic analysis (Sec. 2; Sec. 5.1; Sec. 5.2; the ordering and symbolic steps of Alg. 1 and Alg. 5).
//
// * Without coordinates (general CSR input), nested dissection by graph level
//   structures (Sec. 2): a set of more than leaf_size vertices is split by a
//   breadth-first search (restricted to the set, neighbours in increasing index)
//   from a pseudo-peripheral vertex (the smallest vertex of the last level of a
//   search from the set's smallest vertex); the separator is the first level
//   at which the levels so far hold at least half of the reached vertices
//   (kept between the first and the last level), the lower levels form the first
//   child and the higher levels plus any unreached vertices the second.  Fronts
//   list their vertices in increasing index; a compressed separator is ordered
//   by a breadth-first search of its own subgraph and clustered in balanced
//   halves of that order.
// * Nested dissection by planar separators on integer lattice boxes.  A box is
//   half-open [lo, hi) per axis.  The separator axis is the first axis of
//   largest extent (x, then y, then z); for the node lattice the extent is
//   hi - lo and the plane is lo + ext/2; for the Yee edge lattice (doubled
//   coordinates) the extent counts cells, (hi - lo + 1)/2, and the plane is the
//   node plane (lo - 1) + 2 (ext/2).  Children are [lo, mid) then [mid+1, hi);
//   empty children are dropped; boxes with at most leaf_size unknowns are leaf
//   fronts.  Fronts are numbered in post-order (lower, upper, separator).
// * Inside a front, unknowns are in (z, y, x) lexicographic order; separators
//   with at least nmin_sep unknowns are reordered by recursive geometric
//   bisection (P-hat, Sec. 5.1), giving the HOD-BF cluster tree.
// * I^u = (adj(I^s) U children's I^u) \ subtree, sorted (Sec. 2).
// * F22 cluster tree: balanced halves of the sorted I^u (Sec. 5.1).
// * Nearest neighbours by breadth-first search (Sec. 5.2).
#include "analysis.h"

#include <algorithm>
#include <array>
#include <functional>
#include <numeric>
#include <stdexcept>

namespace mf {

std::vector<std::vector<Range>> cluster_tree_balanced(int64_t npts, int64_t leaf);

namespace {

using C3 = std::array<int64_t, 3>;

struct Builder {
  const int32_t* coords;
  int lattice;
  int leaf, nmin, hleaf;
  bool hybrid = false;
  int par_levels = 0;    // top levels cut along the root's axis (parallel separators)
  int root_axis = 0;
  // graph mode: adjacency with sorted neighbour lists, set membership marks
  std::vector<int64_t> adj_ptr;
  std::vector<int32_t> adj;
  std::vector<int64_t> mark;   // mark[v] == tag: v in the current set
  int64_t tag = 0;
  struct Raw {
    std::vector<int64_t> sep;  // old ids in front order
    std::vector<int64_t> kids;
    bool compressed;
    std::vector<std::vector<Range>> th;
  };
  std::vector<Raw> raw;

  C3 co(int64_t id) const {
    return {coords[3 * id], coords[3 * id + 1], coords[3 * id + 2]};
  }
  bool lex_less(int64_t p, int64_t q) const {
    C3 a = co(p), b = co(q);
    if (a[2] != b[2]) return a[2] < b[2];
    if (a[1] != b[1]) return a[1] < b[1];
    return a[0] < b[0];
  }
  void lex_sort(std::vector<int64_t>& v) const {
    std::sort(v.begin(), v.end(), [this](int64_t p, int64_t q) { return lex_less(p, q); });
  }

  // Recursive geometric bisection with uniform depth (Sec. 5.1).  pts are
  // old ids already in lexicographic order; returns the reordered ids.
  std::vector<int64_t> cluster(const std::vector<int64_t>& pts, std::vector<std::vector<Range>>& levels) const {
    std::vector<std::vector<int64_t>> clusters{pts};
    std::vector<std::vector<std::vector<int64_t>>> hist{clusters};
    auto maxsize = [](const std::vector<std::vector<int64_t>>& cs) {
      size_t m = 0;
      for (auto& c : cs) m = std::max(m, c.size());
      return m;
    };
    while ((int64_t)maxsize(clusters) > hleaf) {
      std::vector<std::vector<int64_t>> nw;
      for (auto& c : clusters) {
        if (c.empty()) { nw.emplace_back(); nw.emplace_back(); continue; }
        C3 lo = co(c[0]), hi = co(c[0]);
        for (int64_t id : c) {
          C3 p = co(id);
          for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], p[d]); hi[d] = std::max(hi[d], p[d]); }
        }
        int a = 0;
        int64_t best = -1;
        for (int d = 0; d < 3; ++d) {
          int64_t ext = hi[d] - lo[d] + 1;
          if (ext > best) { best = ext; a = d; }
        }
        int64_t cut = lo[a] + best / 2;
        std::vector<int64_t> l, r;
        for (int64_t id : c) (co(id)[a] < cut ? l : r).push_back(id);
        nw.push_back(std::move(l));
        nw.push_back(std::move(r));
      }
      clusters = std::move(nw);
      hist.push_back(clusters);
    }
    levels.clear();
    for (auto& lv : hist) {
      std::vector<Range> rs;
      int64_t p = 0;
      for (auto& c : lv) { rs.push_back({p, p + (int64_t)c.size()}); p += (int64_t)c.size(); }
      levels.push_back(std::move(rs));
    }
    std::vector<int64_t> order;
    for (auto& c : clusters) order.insert(order.end(), c.begin(), c.end());
    return order;
  }

  // breadth-first search from s over the vertices with mark == t; returns the levels
  std::vector<std::vector<int64_t>> bfs_levels(int64_t s, int64_t t, std::vector<int64_t>& seen, int64_t stamp) const {
    std::vector<std::vector<int64_t>> lv{{s}};
    seen[s] = stamp;
    for (;;) {
      std::vector<int64_t> nxt;
      for (int64_t v : lv.back())
        for (int64_t k = adj_ptr[v]; k < adj_ptr[v + 1]; ++k) {
          const int64_t w = adj[k];
          if (mark[w] == t && seen[w] != stamp) {
            seen[w] = stamp;
            nxt.push_back(w);
          }
        }
      if (nxt.empty()) break;
      lv.push_back(std::move(nxt));
    }
    return lv;
  }
  std::vector<int64_t> seen_;
  int64_t stamp_ = 0;

  // HOD-BF order of a graph separator: recursive bisection of its two-hop graph (u ~ v when
  // A(u, v) != 0 or u and v share a neighbour) along the balanced tree th.  A node's vertex set
  // (sorted) is searched breadth-first from its smallest vertex, then again from p = the smallest
  // vertex of the last level; the sequence is the levels from p, each sorted, then the vertices not
  // reached (sorted); the first child takes the first (child size) vertices, the second the rest.
  std::vector<int64_t> sep_order(const std::vector<int64_t>& sep, const std::vector<std::vector<Range>>& th) {
    const int64_t ns = (int64_t)sep.size();
    const int64_t t = ++tag;
    if ((int64_t)loc_.size() < (int64_t)mark.size()) loc_.assign(mark.size(), 0);
    for (int64_t i = 0; i < ns; ++i) { mark[sep[i]] = t; loc_[sep[i]] = i; }
    // two-hop graph in local indices (local order = increasing vertex id)
    std::vector<int64_t> p2(ns + 1, 0);
    std::vector<int64_t> a2;
    std::vector<int64_t> nb;
    for (int64_t i = 0; i < ns; ++i) {
      const int64_t v = sep[i];
      nb.clear();
      for (int64_t k = adj_ptr[v]; k < adj_ptr[v + 1]; ++k) {
        const int64_t x = adj[k];
        if (mark[x] == t) nb.push_back(loc_[x]);
        for (int64_t k2 = adj_ptr[x]; k2 < adj_ptr[x + 1]; ++k2) {
          const int64_t y = adj[k2];
          if (mark[y] == t && y != v) nb.push_back(loc_[y]);
        }
      }
      std::sort(nb.begin(), nb.end());
      nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
      a2.insert(a2.end(), nb.begin(), nb.end());
      p2[i + 1] = (int64_t)a2.size();
    }
    std::vector<int64_t> in(ns, 0), seen(ns, 0);
    int64_t in_tag = 0, seen_tag = 0;
    auto levels_from = [&](int64_t s0, int64_t it, int64_t st) {
      std::vector<std::vector<int64_t>> lv{{s0}};
      seen[s0] = st;
      for (;;) {
        std::vector<int64_t> nxt;
        for (int64_t v : lv.back())
          for (int64_t k = p2[v]; k < p2[v + 1]; ++k) {
            const int64_t x = a2[k];
            if (in[x] == it && seen[x] != st) { seen[x] = st; nxt.push_back(x); }
          }
        if (nxt.empty()) break;
        lv.push_back(std::move(nxt));
      }
      return lv;
    };
    std::vector<int64_t> out;
    out.reserve(ns);
    // explicit recursion over (vertex set, level, node)
    std::function<void(std::vector<int64_t>&, size_t, size_t)> order = [&](std::vector<int64_t>& vs, size_t lvl,
                                                                            size_t k) {
      if (lvl + 1 == th.size()) { out.insert(out.end(), vs.begin(), vs.end()); return; }
      const int64_t h = th[lvl + 1][2 * k].b - th[lvl + 1][2 * k].a;
      std::vector<int64_t> left, right;
      if (!vs.empty()) {
        const int64_t it = ++in_tag;
        for (int64_t v : vs) in[v] = it;
        auto lv0 = levels_from(vs[0], it, ++seen_tag);
        const int64_t p = *std::min_element(lv0.back().begin(), lv0.back().end());
        const int64_t st = ++seen_tag;
        auto lv = levels_from(p, it, st);
        std::vector<int64_t> seq;
        seq.reserve(vs.size());
        for (auto& l : lv) {
          std::sort(l.begin(), l.end());
          seq.insert(seq.end(), l.begin(), l.end());
        }
        for (int64_t v : vs)
          if (seen[v] != st) seq.push_back(v);
        const int64_t hh = std::min<int64_t>(h, (int64_t)seq.size());
        left.assign(seq.begin(), seq.begin() + hh);
        right.assign(seq.begin() + hh, seq.end());
        std::sort(left.begin(), left.end());
        std::sort(right.begin(), right.end());
      }
      std::vector<int64_t>().swap(vs);
      order(left, lvl + 1, 2 * k);
      order(right, lvl + 1, 2 * k + 1);
    };
    std::vector<int64_t> all(ns);
    std::iota(all.begin(), all.end(), 0);
    order(all, 0, 0);
    for (auto& v : out) v = sep[v];
    return out;
  }
  std::vector<int64_t> loc_;

  int64_t nd_graph(std::vector<int64_t>& ids) {   // ids sorted ascending
    auto leaf_front = [&](std::vector<int64_t>& v) {
      Raw r;
      r.sep = std::move(v);
      r.compressed = false;
      raw.push_back(std::move(r));
      return (int64_t)raw.size() - 1;
    };
    if ((int64_t)ids.size() <= leaf) return leaf_front(ids);
    const int64_t t = ++tag;
    for (int64_t v : ids) mark[v] = t;
    auto lv0 = bfs_levels(ids[0], t, seen_, ++stamp_);
    const int64_t p = *std::min_element(lv0.back().begin(), lv0.back().end());
    auto lv = bfs_levels(p, t, seen_, ++stamp_);
    const int64_t nl = (int64_t)lv.size();
    if (nl < 3) return leaf_front(ids);   // no level strictly inside the structure
    int64_t reached = 0;
    for (auto& l : lv) reached += (int64_t)l.size();
    int64_t m = 0, acc = 0;
    for (; m < nl; ++m) {
      acc += (int64_t)lv[m].size();
      if (2 * acc >= reached) break;
    }
    m = std::max<int64_t>(1, std::min<int64_t>(m, nl - 2));
    std::vector<int64_t> left, right, sep = lv[m];
    const int64_t st = stamp_;   // seen_[v] == st: v reached from p
    for (int64_t i = 0; i < m; ++i) left.insert(left.end(), lv[i].begin(), lv[i].end());
    for (int64_t i = m + 1; i < nl; ++i) right.insert(right.end(), lv[i].begin(), lv[i].end());
    for (int64_t v : ids)
      if (seen_[v] != st) right.push_back(v);
    std::vector<int64_t>().swap(ids);
    std::sort(left.begin(), left.end());
    std::sort(right.begin(), right.end());
    std::sort(sep.begin(), sep.end());
    std::vector<int64_t> kids;
    if (!left.empty()) kids.push_back(nd_graph(left));
    if (!right.empty()) kids.push_back(nd_graph(right));
    Raw r;
    r.compressed = (int64_t)sep.size() >= nmin;
    if (r.compressed) {
      r.th = cluster_tree_balanced((int64_t)sep.size(), hleaf);
      r.sep = sep_order(sep, r.th);
    } else {
      r.sep = std::move(sep);
    }
    r.kids = std::move(kids);
    raw.push_back(std::move(r));
    return (int64_t)raw.size() - 1;
  }

  int64_t nd(std::vector<int64_t>& ids, C3 lo, C3 hi, int depth = 0) {
    if ((int64_t)ids.size() <= leaf) {
      Raw r;
      r.sep = ids;
      lex_sort(r.sep);
      r.compressed = false;
      raw.push_back(std::move(r));
      return (int64_t)raw.size() - 1;
    }
    C3 ext;
    for (int d = 0; d < 3; ++d) ext[d] = lattice == LATTICE_NODE ? hi[d] - lo[d] : (hi[d] - lo[d] + 1) / 2;
    int a = 0;
    for (int d = 1; d < 3; ++d)
      if (ext[d] > ext[a]) a = d;
    if (depth == 0) root_axis = a;
    else if (depth < par_levels && ext[root_axis] >= 3) a = root_axis;   // parallel to the root separator
    int64_t mid = lattice == LATTICE_NODE ? lo[a] + ext[a] / 2 : (lo[a] - 1) + 2 * (ext[a] / 2);
    if (hybrid) {
      // a box whose planar separator would stay dense is ordered by graph nested dissection
      int64_t ns = 0;
      for (int64_t id : ids) ns += coords[3 * id + a] == mid;
      if (ns < nmin) {
        std::sort(ids.begin(), ids.end());
        return nd_graph(ids);
      }
    }
    std::vector<int64_t> left, right, sep;
    for (int64_t id : ids) {
      int64_t c = coords[3 * id + a];
      if (c < mid) left.push_back(id);
      else if (c > mid) right.push_back(id);
      else sep.push_back(id);
    }
    std::vector<int64_t>().swap(ids);
    std::vector<int64_t> kids;
    if (!left.empty()) {
      C3 h2 = hi; h2[a] = mid;
      kids.push_back(nd(left, lo, h2, depth + 1));
    }
    if (!right.empty()) {
      C3 l2 = lo; l2[a] = mid + 1;
      kids.push_back(nd(right, l2, hi, depth + 1));
    }
    if (sep.empty()) throw std::runtime_error("empty separator: the lattice rule does not apply to this input");
    Raw r;
    lex_sort(sep);
    r.compressed = (int64_t)sep.size() >= nmin;
    if (r.compressed) r.sep = cluster(sep, r.th);
    else r.sep = std::move(sep);
    r.kids = std::move(kids);
    raw.push_back(std::move(r));
    return (int64_t)raw.size() - 1;
  }
};

}  // namespace

std::vector<std::vector<Range>> cluster_tree_balanced(int64_t npts, int64_t leaf) {
  std::vector<std::vector<Range>> lv{{{0, npts}}};
  for (;;) {
    int64_t mx = 0;
    for (auto& r : lv.back()) mx = std::max(mx, r.b - r.a);
    if (mx <= leaf) break;
    std::vector<Range> nw;
    for (auto& r : lv.back()) {
      int64_t m = r.a + (r.b - r.a + 1) / 2;
      nw.push_back({r.a, m});
      nw.push_back({m, r.b});
    }
    lv.push_back(std::move(nw));
  }
  return lv;
}

void analyze(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* coords, int lattice,
             int leaf_size, int nmin_sep, int hodbf_leaf, Analysis& out, int ordering, int parallel_levels) {
  if (parallel_levels < 0) throw std::runtime_error("parallel_levels must be >= 0");
  if (ordering != ORDER_AUTO && ordering != ORDER_HYBRID && ordering != ORDER_GRAPH)
    throw std::runtime_error("unknown ordering");
  if (ordering == ORDER_HYBRID && !coords) throw std::runtime_error("the hybrid ordering needs lattice coordinates");
  if (n <= 0 || !rowptr || !colind) throw std::runtime_error("invalid CSR");
  if (lattice != LATTICE_NODE && lattice != LATTICE_EDGE) throw std::runtime_error("unknown lattice");
  if (leaf_size < 1 || hodbf_leaf < 1 || nmin_sep < 1) throw std::runtime_error("invalid sizes in options");
  if (rowptr[0] != 0) throw std::runtime_error("rowptr[0] must be 0");
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) throw std::runtime_error("rowptr not monotone");
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (colind[k] < 0 || colind[k] >= n) throw std::runtime_error("column index out of range");
  }
  Builder b;
  // sorted off-diagonal neighbour lists; the pattern must be structurally symmetric
  b.adj_ptr.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    std::vector<int32_t> nb;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (colind[k] != i) nb.push_back(colind[k]);
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    b.adj.insert(b.adj.end(), nb.begin(), nb.end());
    b.adj_ptr[i + 1] = (int64_t)b.adj.size();
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = b.adj_ptr[i]; k < b.adj_ptr[i + 1]; ++k) {
      const int64_t j = b.adj[k];
      if (!std::binary_search(b.adj.begin() + b.adj_ptr[j], b.adj.begin() + b.adj_ptr[j + 1], (int32_t)i))
        throw std::runtime_error("pattern not structurally symmetric");
    }
  b.coords = coords;
  b.lattice = lattice;
  b.leaf = leaf_size;
  b.nmin = nmin_sep;
  b.hleaf = hodbf_leaf;
  b.hybrid = ordering == ORDER_HYBRID;
  b.par_levels = parallel_levels;
  b.mark.assign(n, 0);
  b.seen_.assign(n, 0);
  if (!coords || ordering == ORDER_GRAPH) {
    std::vector<int64_t> all(n);
    std::iota(all.begin(), all.end(), 0);
    b.nd_graph(all);
  } else {
  C3 mn{INT64_MAX, INT64_MAX, INT64_MAX}, mx{INT64_MIN, INT64_MIN, INT64_MIN};
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      mn[d] = std::min<int64_t>(mn[d], coords[3 * i + d]);
      mx[d] = std::max<int64_t>(mx[d], coords[3 * i + d]);
    }
  C3 lo, hi;
  for (int d = 0; d < 3; ++d) {
    if (lattice == LATTICE_NODE) { lo[d] = mn[d]; hi[d] = mx[d] + 1; }
    else {
      if (mn[d] < 1) throw std::runtime_error("edge lattice coordinates must be positive");
      lo[d] = 2 * ((mn[d] - 1) / 2) + 1;
      hi[d] = 2 * (mx[d] / 2 + 1);
    }
  }
  std::vector<int64_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  b.nd(all, lo, hi);
  }

  out = Analysis();
  out.n = n;
  out.leaf_size = leaf_size;
  out.nmin_sep = nmin_sep;
  out.hodbf_leaf = hodbf_leaf;
  out.perm.reserve(n);
  out.fronts.resize(b.raw.size());
  int64_t pos = 0;
  for (size_t f = 0; f < b.raw.size(); ++f) {
    auto& r = b.raw[f];
    FrontInfo& fi = out.fronts[f];
    fi.id = (int64_t)f;
    fi.children = r.kids;
    fi.sep_begin = pos;
    fi.sep_end = pos + (int64_t)r.sep.size();
    fi.sub_begin = pos;
    fi.compressed = r.compressed;
    fi.th_tree = r.th;
    pos = fi.sep_end;
    out.perm.insert(out.perm.end(), r.sep.begin(), r.sep.end());
  }
  if ((int64_t)out.perm.size() != n) throw std::runtime_error("nested dissection lost unknowns");
  out.iperm.assign(n, -1);
  for (int64_t i = 0; i < n; ++i) out.iperm[out.perm[i]] = i;
  for (auto& f : out.fronts)
    for (int64_t c : f.children) out.fronts[c].parent = f.id;
  for (auto& f : out.fronts)
    for (int64_t c : f.children) f.sub_begin = std::min(f.sub_begin, out.fronts[c].sub_begin);
  // permuted pattern
  out.prow.assign(n + 1, 0);
  for (int64_t r = 0; r < n; ++r) {
    int64_t o = out.perm[r];
    out.prow[r + 1] = out.prow[r] + (rowptr[o + 1] - rowptr[o]);
  }
  out.pcol.resize(out.prow[n]);
  for (int64_t r = 0; r < n; ++r) {
    int64_t o = out.perm[r];
    int64_t p = out.prow[r];
    for (int64_t k = rowptr[o]; k < rowptr[o + 1]; ++k) out.pcol[p++] = out.iperm[colind[k]];
    std::sort(out.pcol.begin() + out.prow[r], out.pcol.begin() + out.prow[r + 1]);
  }
  // symbolic factorization
  for (auto& f : out.fronts) {
    std::vector<int64_t> cand;
    for (int64_t r = f.sep_begin; r < f.sep_end; ++r)
      cand.insert(cand.end(), out.pcol.begin() + out.prow[r], out.pcol.begin() + out.prow[r + 1]);
    for (int64_t c : f.children) cand.insert(cand.end(), out.fronts[c].upd.begin(), out.fronts[c].upd.end());
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (int64_t g : cand)
      if (g >= f.sep_end) f.upd.push_back(g);
    if (f.compressed) f.f22_tree = cluster_tree_balanced(f.u(), hodbf_leaf);
  }
  for (int64_t i = (int64_t)out.fronts.size() - 1; i >= 0; --i) {
    auto& f = out.fronts[i];
    f.level = f.parent < 0 ? 0 : out.fronts[f.parent].level + 1;
  }
}

void bfs_nearest(const Analysis& an, int64_t start, const std::vector<uint8_t>& allowed,
                 const std::vector<uint8_t>& target, int knn, std::vector<int64_t>& out,
                 std::vector<int64_t>& stamp, int64_t& stamp_val) {
  out.clear();
  ++stamp_val;
  stamp[start] = stamp_val;
  std::vector<int64_t> frontier{start}, nxt;
  while (!frontier.empty() && (int)out.size() < knn) {
    nxt.clear();
    for (int64_t v : frontier)
      for (int64_t k = an.prow[v]; k < an.prow[v + 1]; ++k) {
        int64_t w = an.pcol[k];
        if (allowed[w] && stamp[w] != stamp_val) { stamp[w] = stamp_val; nxt.push_back(w); }
      }
    std::sort(nxt.begin(), nxt.end());
    for (int64_t w : nxt)
      if (target[w]) {
        out.push_back(w);
        if ((int)out.size() == knn) break;
      }
    frontier.swap(nxt);
  }
}

void front_neighbours(const Analysis& an, const FrontInfo& f, int knn, FrontNeighbours& o) {
  const int64_t N = an.n;
  std::vector<uint8_t> in_s(N, 0), in_u(N, 0), both(N, 0), tgt(N, 0);
  for (int64_t g = f.sep_begin; g < f.sep_end; ++g) in_s[g] = both[g] = 1;
  for (int64_t g : f.upd) in_u[g] = both[g] = 1;
  std::vector<int64_t> stamp(N, 0), res;
  int64_t sv = 0;
  std::vector<int64_t> leaf_of(N, -1), leaf22(N, -1);
  if (!f.th_tree.empty()) {
    auto& lv = f.th_tree.back();
    for (size_t li = 0; li < lv.size(); ++li)
      for (int64_t p = lv[li].a; p < lv[li].b; ++p) leaf_of[f.sep_begin + p] = (int64_t)li;
  } else {
    for (int64_t g = f.sep_begin; g < f.sep_end; ++g) leaf_of[g] = 0;
  }
  if (!f.f22_tree.empty()) {
    auto& lv = f.f22_tree.back();
    for (size_t li = 0; li < lv.size(); ++li)
      for (int64_t p = lv[li].a; p < lv[li].b; ++p) leaf22[f.upd[p]] = (int64_t)li;
  } else {
    for (int64_t g : f.upd) leaf22[g] = 0;
  }
  auto run = [&](const std::vector<int64_t>& verts, const std::vector<uint8_t>& allowed,
                 const std::function<bool(int64_t, int64_t)>& is_target, std::vector<int64_t>& ptr,
                 std::vector<int64_t>& idx) {
    ptr.assign(1, 0);
    idx.clear();
    for (int64_t x : verts) {
      res.clear();
      // BFS with a per-start target predicate
      ++sv;
      stamp[x] = sv;
      std::vector<int64_t> frontier{x}, nxt;
      while (!frontier.empty() && (int)res.size() < knn) {
        nxt.clear();
        for (int64_t v : frontier)
          for (int64_t k = an.prow[v]; k < an.prow[v + 1]; ++k) {
            int64_t w = an.pcol[k];
            if (allowed[w] && stamp[w] != sv) { stamp[w] = sv; nxt.push_back(w); }
          }
        std::sort(nxt.begin(), nxt.end());
        for (int64_t w : nxt)
          if (is_target(x, w)) {
            res.push_back(w);
            if ((int)res.size() == knn) break;
          }
        frontier.swap(nxt);
      }
      idx.insert(idx.end(), res.begin(), res.end());
      ptr.push_back((int64_t)idx.size());
    }
  };
  std::vector<int64_t> sv_list, uv_list(f.upd);
  for (int64_t g = f.sep_begin; g < f.sep_end; ++g) sv_list.push_back(g);
  run(sv_list, in_s, [&](int64_t x, int64_t w) { return in_s[w] && leaf_of[w] != leaf_of[x]; }, o.nn11_ptr, o.nn11);
  run(uv_list, in_u, [&](int64_t x, int64_t w) { return in_u[w] && leaf22[w] != leaf22[x]; }, o.nn22_ptr, o.nn22);
  run(sv_list, both, [&](int64_t, int64_t w) { return (bool)in_u[w]; }, o.nn12_ptr, o.nn12);
  run(uv_list, both, [&](int64_t, int64_t w) { return (bool)in_s[w]; }, o.nn21_ptr, o.nn21);
}

}  // namespace mf
