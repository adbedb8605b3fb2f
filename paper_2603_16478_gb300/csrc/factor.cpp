// Host-side factorisation of the scalar elastic matrix A_s (A = A_s (x) I_3).
//
// The paper's forward solver keeps a Cholesky factor A = L L^T and its explicit sparse
// inverse S = L^{-1}, so that A^{-1} = S^T S is two sparse matrix-vector products
// (Sec. 3, "GPU acceleration via sparse-inverse factorization").  This file computes, once
// per scene:
//   1. a nested-dissection ordering from the vertex coordinates (recursive median
//      bisection along the longest axis with one-sided vertex separators, separators last),
//   2. the elimination tree of the permuted matrix,
//   3. the Cholesky factor by the up-looking row-by-row algorithm (each row of L is a
//      sparse triangular solve whose pattern is the row's reach in the elimination tree),
//   4. the columns of S = L^{-1}: column j is nonzero exactly on the elimination-tree path
//      from j to its root, and is obtained by a forward substitution along that path.
#include <algorithm>
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
  for (int v = 0; v < n; ++v) {
    int k = F.iperm[v];
    for (int64_t p = As.ptr[v]; p < As.ptr[v + 1]; ++p) {
      int i = F.iperm[As.col[p]];
      if (i <= k) upper[k].push_back({i, As.val[p]});
    }
  }
  // 2. elimination tree (with path compression through `anc`)
  F.parent.assign(n, -1);
  {
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
  }
  // 3. up-looking Cholesky: row k of L solves L(0:k,0:k) y = A(0:k, k)
  std::vector<std::vector<std::pair<int, double>>> Lcol(n);  // strictly-lower entries (row, val)
  std::vector<double> Ldiag(n);
  {
    std::vector<double> x(n, 0.0);
    std::vector<int32_t> mark(n, -1), reach;
    for (int k = 0; k < n; ++k) {
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
      if (!(d > 0.0)) throw Error{NCPADJ_ERR_INVALID_ARG, "elastic matrix is not positive definite"};
      Ldiag[k] = std::sqrt(d);
    }
  }
  F.nnz_L = n;
  for (int j = 0; j < n; ++j) F.nnz_L += (int64_t)Lcol[j].size();
  // 4. columns of S = L^{-1} along the elimination-tree paths
  {
    std::vector<double> x(n, 0.0);
    std::vector<int32_t> path;
    F.St.n = n;
    F.St.ptr.assign(n + 1, 0);
    std::vector<std::vector<std::pair<int, double>>> cols(n);
    int64_t total = 0;
    for (int j = 0; j < n; ++j) {
      path.clear();
      for (int i = j; i != -1; i = F.parent[i]) path.push_back(i);
      x[j] = 1.0;
      for (int i : path) {
        x[i] /= Ldiag[i];
        double xi = x[i];
        for (auto& e : Lcol[i]) x[e.first] -= e.second * xi;
      }
      total += (int64_t)path.size();
      F.St.ptr[j + 1] = total;
      for (int i : path) {
        F.St.col.push_back(i);
        F.St.val.push_back(x[i]);
        x[i] = 0.0;
      }
    }
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
