// Host-side factorisation of the scalar elastic matrix A_s (A = A_s (x) I_3).
//
// The paper's forward solver keeps a Cholesky factor A = L L^T and its explicit sparse
// inverse S = L^{-1}, so that A^{-1} = S^T S is two sparse matrix-vector products
// (Sec. 3, "GPU acceleration via sparse-inverse factorization").  This file computes, once
// per scene:
//   1. a nested-dissection ordering from the vertex coordinates (recursive median
//      bisection along the longest axis with one-sided vertex separators, separators last),
//   2. the elimination tree of the permuted matrix, and the ordering refined to a postorder of
//      that tree (an equivalent ordering: the same fill and the same tree, relabelled so that
//      every subtree is a contiguous range of positions ending at its root),
//   3. the Cholesky factor by the up-looking row-by-row algorithm (each row of L is a
//      sparse triangular solve whose pattern is the row's reach in the elimination tree),
//   4. the columns of S = L^{-1}: column j is nonzero exactly on the elimination-tree path
//      from j to its root, and is obtained by a forward substitution along that path.  So row i
//      of S holds exactly the descendants of i: in the postorder, the contiguous range
//      [i - size(i) + 1, i].
#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <numeric>
#include <stdexcept>

#include "internal.h"

namespace ncpadj {

namespace {

struct Graph {
  int n;
  const CsrD* A;
};

void nd_recurse(const CsrD& A, const double* xyz, std::vector<int32_t>& verts, std::vector<int32_t>& side,
                int level_tag, std::vector<int32_t>& order) {
  const size_t kLeaf = 64;
  if (verts.size() <= kLeaf) {
    order.insert(order.end(), verts.begin(), verts.end());
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v : verts)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], xyz[3 * v + d]);
      hi[d] = std::max(hi[d], xyz[3 * v + d]);
    }
  int axis = 0;
  for (int d = 1; d < 3; ++d)
    if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
  size_t mid = verts.size() / 2;
  std::nth_element(verts.begin(), verts.begin() + mid, verts.end(), [&](int a, int b) {
    double xa = xyz[3 * a + axis], xb = xyz[3 * b + axis];
    return xa < xb || (xa == xb && a < b);
  });
  // mark the right half with a tag unique to this call
  for (size_t i = mid; i < verts.size(); ++i) side[verts[i]] = level_tag;
  std::vector<int32_t> left, right, sep;
  for (size_t i = 0; i < mid; ++i) {
    int v = verts[i];
    bool touches = false;
    for (int64_t p = A.ptr[v]; p < A.ptr[v + 1] && !touches; ++p) touches = side[A.col[p]] == level_tag;
    (touches ? sep : left).push_back(v);
  }
  right.assign(verts.begin() + mid, verts.end());
  for (int v : right) side[v] = -1;
  if (left.empty() || right.empty()) {  // degenerate split: stop recursing
    order.insert(order.end(), verts.begin(), verts.end());
    return;
  }
  std::vector<int32_t>().swap(verts);
  nd_recurse(A, xyz, left, side, 2 * level_tag, order);
  nd_recurse(A, xyz, right, side, 2 * level_tag + 1, order);
  order.insert(order.end(), sep.begin(), sep.end());
}

}  // namespace

void factor_elastic(const CsrD& As, const double* xyz, ElasticFactor& F) {
  const int n = As.n;
  F.n = n;
  // 1. ordering
  {
    std::vector<int32_t> verts(n), side(n, -1), order;
    std::iota(verts.begin(), verts.end(), 0);
    order.reserve(n);
    nd_recurse(As, xyz, verts, side, 1, order);
    if ((int)order.size() != n) throw Error{NCPADJ_ERR_INVALID_ARG, "ordering lost vertices"};
    F.perm = order;
    F.iperm.assign(n, -1);
    for (int i = 0; i < n; ++i) F.iperm[F.perm[i]] = i;
  }
  // permuted matrix, upper part by columns: for column k, rows i <= k with A(i,k) != 0
  std::vector<std::vector<std::pair<int, double>>> upper(n);
  auto permute = [&]() {
    for (auto& u : upper) u.clear();
    for (int v = 0; v < n; ++v) {
      int k = F.iperm[v];
      for (int64_t p = As.ptr[v]; p < As.ptr[v + 1]; ++p) {
        int i = F.iperm[As.col[p]];
        if (i <= k) upper[k].push_back({i, As.val[p]});
      }
    }
  };
  // 2. elimination tree (with path compression through `anc`)
  auto etree = [&]() {
    F.parent.assign(n, -1);
    std::vector<int32_t> anc(n, -1);
    for (int k = 0; k < n; ++k) {
      for (auto& e : upper[k]) {
        int i = e.first;
        while (i != -1 && i < k) {
          int next = anc[i];
          anc[i] = k;
          if (next == -1) {
            F.parent[i] = k;
            break;
          }
          i = next;
        }
      }
    }
  };
  permute();
  etree();
  // postorder of the forest (roots and children in increasing position), then the same tree in
  // that numbering: position k of the new ordering is node post[k] of the old one
  {
    std::vector<int32_t> first(n, -1), next(n, -1), post;
    post.reserve(n);
    for (int j = n - 1; j >= 0; --j)  // child lists in increasing order
      if (F.parent[j] >= 0) {
        next[j] = first[F.parent[j]];
        first[F.parent[j]] = j;
      }
    std::vector<int32_t> stack;
    for (int r = 0; r < n; ++r) {
      if (F.parent[r] >= 0) continue;
      stack.push_back(r);
      while (!stack.empty()) {
        const int v = stack.back();
        if (first[v] >= 0) {  // descend into the next unvisited child
          const int c = first[v];
          first[v] = next[c];
          stack.push_back(c);
        } else {
          post.push_back(v);
          stack.pop_back();
        }
      }
    }
    if ((int)post.size() != n) throw Error{NCPADJ_ERR_INVALID_ARG, "postorder lost nodes"};
    std::vector<int32_t> perm(n);
    for (int k = 0; k < n; ++k) perm[k] = F.perm[post[k]];
    F.perm = perm;
    for (int i = 0; i < n; ++i) F.iperm[F.perm[i]] = i;
    permute();
    etree();
  }
  // 3. up-looking Cholesky: row k of L solves L(0:k,0:k) y = A(0:k, k).  Row k reads and
  // appends to columns of k's descendants only, so the rows of disjoint elimination subtrees are
  // independent: subtrees of about n/(8 threads) nodes are factored in parallel (each in
  // increasing row order), then the remaining top nodes (separators) in increasing order.  Every
  // row sees exactly the data it sees in a serial sweep: the result is bit-identical.
  std::vector<std::vector<std::pair<int, double>>> Lcol(n);  // strictly-lower entries (row, val)
  std::vector<double> Ldiag(n);
  std::atomic<bool> indefinite{false};
  auto factor_rows = [&](const std::vector<int32_t>& rows, std::vector<double>& x, std::vector<int32_t>& mark,
                         std::vector<int32_t>& reach) {
    for (int k : rows) {
      reach.clear();
      mark[k] = k;
      double akk = 0.0;
      for (auto& e : upper[k]) {
        if (e.first == k) {
          akk += e.second;
          continue;
        }
        x[e.first] += e.second;
        for (int i = e.first; i != -1 && mark[i] != k; i = F.parent[i]) {
          mark[i] = k;
          reach.push_back(i);
        }
      }
      std::sort(reach.begin(), reach.end());  // ancestors carry larger positions
      double d = akk;
      for (int j : reach) {
        double y = x[j] / Ldiag[j];
        x[j] = 0.0;
        for (auto& e : Lcol[j]) x[e.first] -= e.second * y;  // rows < k of column j
        d -= y * y;
        Lcol[j].push_back({k, y});
      }
      if (!(d > 0.0)) {
        indefinite = true;
        d = 1.0;
      }
      Ldiag[k] = std::sqrt(d);
    }
  };
  const int nthreads = std::max(1, std::min<int>(64, (int)std::thread::hardware_concurrency()));
  {
    std::vector<std::vector<int32_t>> children(n);
    std::vector<int32_t> size(n, 1), roots;
    for (int j = 0; j < n; ++j) {
      if (F.parent[j] < 0) roots.push_back(j);
      else children[F.parent[j]].push_back(j);
    }
    for (int j = 0; j < n; ++j)
      if (F.parent[j] >= 0) size[F.parent[j]] += size[j];  // parent > j: sizes complete in order
    const int target = std::max(256, n / (8 * nthreads));
    std::vector<int32_t> top, stack(roots.begin(), roots.end());
    std::vector<std::vector<int32_t>> tasks;
    while (!stack.empty()) {
      const int r = stack.back();
      stack.pop_back();
      if (size[r] > target && !children[r].empty()) {
        top.push_back(r);
        for (int c : children[r]) stack.push_back(c);
      } else {
        std::vector<int32_t> rows, st2{r};
        while (!st2.empty()) {
          const int v = st2.back();
          st2.pop_back();
          rows.push_back(v);
          for (int c : children[v]) st2.push_back(c);
        }
        std::sort(rows.begin(), rows.end());
        tasks.push_back(std::move(rows));
      }
    }
    std::sort(tasks.begin(), tasks.end(), [](const auto& a, const auto& b) { return a.size() > b.size(); });
    std::atomic<size_t> next{0};
    auto worker = [&]() {
      std::vector<double> x(n, 0.0);
      std::vector<int32_t> mark(n, -1), reach;
      for (size_t t; (t = next.fetch_add(1)) < tasks.size();) factor_rows(tasks[t], x, mark, reach);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < std::min<int>(nthreads, (int)tasks.size()); ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    std::sort(top.begin(), top.end());
    std::vector<double> x(n, 0.0);
    std::vector<int32_t> mark(n, -1), reach;
    factor_rows(top, x, mark, reach);
  }
  if (indefinite) throw Error{NCPADJ_ERR_INVALID_ARG, "elastic matrix is not positive definite"};
  F.nnz_L = n;
  for (int j = 0; j < n; ++j) F.nnz_L += (int64_t)Lcol[j].size();
  // 4. columns of S = L^{-1} along the elimination-tree paths.  Column j has one entry per node of
  // the path from j to its root, so the layout is known up front; the columns are independent
  // and are computed by all host threads, each with its own dense work vector.
  {
    F.St.n = n;
    F.St.ptr.assign(n + 1, 0);
    std::vector<int32_t> depth(n, 0);
    for (int j = n - 1; j >= 0; --j) depth[j] = F.parent[j] < 0 ? 1 : depth[F.parent[j]] + 1;  // parent > j
    for (int j = 0; j < n; ++j) F.St.ptr[j + 1] = F.St.ptr[j] + depth[j];
    const int64_t total = F.St.ptr[n];
    F.St.col.assign(total, 0);
    F.St.val.assign(total, 0.0);
    std::atomic<int> next{0};
    auto worker = [&]() {
      std::vector<double> x(n, 0.0);
      for (;;) {
        const int j0 = next.fetch_add(64);
        if (j0 >= n) break;
        for (int j = j0; j < std::min(n, j0 + 64); ++j) {
          int64_t p = F.St.ptr[j];
          x[j] = 1.0;
          for (int i = j; i != -1; i = F.parent[i]) {
            x[i] /= Ldiag[i];
            const double xi = x[i];
            for (auto& e : Lcol[i]) x[e.first] -= e.second * xi;
            F.St.col[p] = i;
            F.St.val[p] = xi;
            x[i] = 0.0;
            ++p;
          }
        }
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    // S by rows (transpose of St)
    F.S.n = n;
    F.S.ptr.assign(n + 1, 0);
    for (int64_t p = 0; p < total; ++p) F.S.ptr[F.St.col[p] + 1]++;
    for (int i = 0; i < n; ++i) F.S.ptr[i + 1] += F.S.ptr[i];
    F.S.col.assign(total, 0);
    F.S.val.assign(total, 0.0);
    std::vector<int64_t> fill(F.S.ptr.begin(), F.S.ptr.end() - 1);
    for (int j = 0; j < n; ++j)
      for (int64_t p = F.St.ptr[j]; p < F.St.ptr[j + 1]; ++p) {
        int i = F.St.col[p];
        F.S.col[fill[i]] = j;
        F.S.val[fill[i]] = F.St.val[p];
        fill[i]++;
      }
  }
}

}  // namespace ncpadj
