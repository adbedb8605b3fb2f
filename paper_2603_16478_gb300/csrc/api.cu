// C-ABI entry points, scene set-up and the host-driven adjoint solve.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace ncpadj {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

void DevBuf::ensure(size_t n) {
  if (n <= bytes) return;
  release();
  if (n == 0) return;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    bytes = 0;
    cudaGetLastError();
    throw Error{NCPADJ_ERR_OOM, "cudaMalloc of " + std::to_string(n) + " bytes failed"};
  }
  bytes = n;
}
void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

template <class T>
static void upload(DevBuf& b, const std::vector<T>& v) {
  b.ensure(std::max<size_t>(v.size() * sizeof(T), 16));
  if (!v.empty()) NCPADJ_CUDA_TRY(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// Chunks of the rows of S and S^T for the A^{-1} product: at most len entries each (one warp per
// chunk, len / 32 values per lane), with S's first column per chunk (its rows are column ranges)
static void rechunk(Scene& S, int len) {
  auto chunk = [len](const std::vector<int64_t>& ptr, int n, DevBuf& crow, DevBuf& cb, DevBuf& ce) {
    std::vector<int32_t> r;
    std::vector<int64_t> b, e;
    for (int i = 0; i < n; ++i)
      for (int64_t p = ptr[i]; p < ptr[i + 1]; p += len) {
        r.push_back(i);
        b.push_back(p);
        e.push_back(std::min<int64_t>(p + len, ptr[i + 1]));
      }
    upload(crow, r);
    upload(cb, b);
    upload(ce, e);
    return (int)r.size();
  };
  const int n = (int)S.S_first_h.size();
  S.nS_chunks = chunk(S.S_ptr_h, n, S.S_crow, S.S_cbeg, S.S_cend);
  std::vector<int32_t> c0;
  c0.reserve(S.nS_chunks);
  for (int i = 0; i < n; ++i)
    for (int64_t p = S.S_ptr_h[i]; p < S.S_ptr_h[i + 1]; p += len)
      c0.push_back(S.S_first_h[i] + (int32_t)(p - S.S_ptr_h[i]));
  upload(S.S_c0, c0);
  S.nSt_chunks = chunk(S.St_ptr_h, n, S.St_crow, S.St_cbeg, S.St_cend);
  S.chunk = len;
}

static ncpadj_status fail(const Error& e) {
  set_error(e.msg);
  return e.status;
}

// ------------------------------------------------------------------------------------------
// scene set-up
// ------------------------------------------------------------------------------------------
// One mesh of a scene: tets (nvpe = 4), or the triangles of a shell (nvpe = 3) with its thickness
// and bending stiffness.
struct MeshSpec {
  int nv = 0, ne = 0, nvpe = 4;
  const double* rest_pos = nullptr;
  const int32_t* elems = nullptr;
  const double* E = nullptr;
  const double* nu = nullptr;
  double density = 0, h = 0, thickness = 0, bend = 0;
};
static MeshSpec spec_of(const ncpadj_scene_desc& d) {
  MeshSpec m;
  m.nv = d.n_verts;
  m.ne = d.n_tets;
  m.rest_pos = d.rest_pos;
  m.elems = d.tets;
  m.E = d.E;
  m.nu = d.nu;
  m.density = d.density;
  m.h = d.h;
  return m;
}
static MeshSpec spec_of(const ncpadj_shell_desc& d) {
  MeshSpec m;
  m.nv = d.n_verts;
  m.ne = d.n_tris;
  m.nvpe = 3;
  m.rest_pos = d.rest_pos;
  m.elems = d.tris;
  m.E = d.E;
  m.nu = d.nu;
  m.density = d.density;
  m.h = d.h;
  m.thickness = d.thickness;
  m.bend = d.bend;
  return m;
}

// One mesh's share of a (batch) scene, computed independently of the others.
struct MeshPart {
  std::vector<double> gvec, vol, mu, lam, lame_d, mass;
  std::vector<int32_t> row_ptr, col, slot, diag_slot;  // local vertex numbering
  std::vector<int32_t> bidx, bslot;                    // bending hinges: vertices [4], slots [16]
  std::vector<double> bcoef;                           // K_0..K_3, 3/(A_1+A_2)
  ElasticFactor F;
  double ms_factor = 0;
};

// Rest operator of tet t: g_a = row (a-1) of D_m^{-1} for a = 1..3, g_0 = -(g_1 + g_2 + g_3), so that
// F = sum_a x_a g_a^T; returns the volume.
static double tet_rest(const double* X, const int v[4], int t, double* g) {
  double Dm[3][3];  // columns X_a - X_0
  for (int a = 1; a < 4; ++a)
    for (int r = 0; r < 3; ++r) Dm[r][a - 1] = X[3 * v[a] + r] - X[3 * v[0] + r];
  double det = Dm[0][0] * (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) -
               Dm[0][1] * (Dm[1][0] * Dm[2][2] - Dm[1][2] * Dm[2][0]) +
               Dm[0][2] * (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]);
  NCPADJ_REQUIRE(det > 0 && std::isfinite(det), "tet " + std::to_string(t) + " is inverted or degenerate at rest");
  double B[3][3];  // inverse by cofactors
  B[0][0] = (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) / det;
  B[0][1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) / det;
  B[0][2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) / det;
  B[1][0] = (Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2]) / det;
  B[1][1] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) / det;
  B[1][2] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) / det;
  B[2][0] = (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]) / det;
  B[2][1] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) / det;
  B[2][2] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) / det;
  for (int k = 0; k < 3; ++k) {
    g[k] = -(B[0][k] + B[1][k] + B[2][k]);
    for (int a = 1; a < 4; ++a) g[3 * a + k] = B[a - 1][k];
  }
  return det / 6.0;
}

static inline void sub3(const double* X, int i, int j, double* out) {
  for (int r = 0; r < 3; ++r) out[r] = X[3 * i + r] - X[3 * j + r];
}
static inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Rest operator of triangle t in its own plane: orthonormal axes a_1 = e_1/|e_1|, a_2 = n x a_1,
// D_m = [a_i . e_j] (2 x 2), g_a = row (a-1) of D_m^{-1} for a = 1, 2, g_0 = -(g_1 + g_2); returns
// the area.
static double tri_rest(const double* X, const int v[3], int t, double* g) {
  double e1[3], e2[3], n[3];
  sub3(X, v[1], v[0], e1);
  sub3(X, v[2], v[0], e2);
  cross3(e1, e2, n);
  const double area2 = std::sqrt(dot3(n, n)), l1 = std::sqrt(dot3(e1, e1));
  NCPADJ_REQUIRE(area2 > 0 && std::isfinite(area2) && l1 > 0,
                 "triangle " + std::to_string(t) + " is degenerate at rest");
  double a1[3], a2[3], nn[3];
  for (int r = 0; r < 3; ++r) {
    a1[r] = e1[r] / l1;
    nn[r] = n[r] / area2;
  }
  cross3(nn, a1, a2);
  const double D00 = dot3(a1, e1), D01 = dot3(a1, e2), D10 = dot3(a2, e1), D11 = dot3(a2, e2);
  const double det = D00 * D11 - D01 * D10;
  const double B[2][2] = {{D11 / det, -D01 / det}, {-D10 / det, D00 / det}};
  for (int k = 0; k < 2; ++k) {
    g[k] = -(B[0][k] + B[1][k]);
    g[2 + k] = B[0][k];
    g[4 + k] = B[1][k];
  }
  return 0.5 * area2;
}

// Isometric bending hinges of a triangle mesh: for every edge (i0, i1) shared by two triangles with
// opposite vertices i2, i3, the cotangent stencil (Bergou et al. 2006)
//   K = (c03 + c04, c01 + c02, -c01 - c03, -c02 - c04),
// c0j the cotangent of the angle at vertex i0 between the edge and (x_ij - x_i0) (j = 2, 3 as c01, c02),
// c1j the same at i1 (as c03, c04), and 3/(A_1 + A_2) with A_1, A_2 the triangles' areas.
static void bending_hinges(const MeshSpec& d, MeshPart& P) {
  const double* X = d.rest_pos;
  std::vector<std::pair<int64_t, int32_t>> he;  // (edge key, opposite vertex)
  he.reserve(3 * (size_t)d.ne);
  for (int t = 0; t < d.ne; ++t) {
    const int32_t* v = d.elems + 3 * (size_t)t;
    for (int k = 0; k < 3; ++k) {
      const int32_t u = v[k], w = v[(k + 1) % 3], o = v[(k + 2) % 3];
      he.push_back({(int64_t)std::min(u, w) * d.nv + std::max(u, w), o});
    }
  }
  std::sort(he.begin(), he.end());
  auto cot = [](const double* p, const double* q) {
    double c[3];
    cross3(p, q, c);
    return dot3(p, q) / std::sqrt(dot3(c, c));
  };
  for (size_t i = 0; i < he.size();) {
    size_t j = i;
    while (j < he.size() && he[j].first == he[i].first) ++j;
    NCPADJ_REQUIRE(j - i <= 2, "an edge is shared by more than two triangles");
    if (j - i == 2) {
      const int i0 = (int)(he[i].first / d.nv), i1 = (int)(he[i].first % d.nv);
      const int i2 = he[i].second, i3 = he[i + 1].second;
      double e0[3], e1[3], e2[3], e3[3], e4[3], m0[3], n1[3], n2[3];
      sub3(X, i1, i0, e0);
      sub3(X, i2, i0, e1);
      sub3(X, i3, i0, e2);
      sub3(X, i2, i1, e3);
      sub3(X, i3, i1, e4);
      for (int r = 0; r < 3; ++r) m0[r] = -e0[r];
      const double c01 = cot(e0, e1), c02 = cot(e0, e2), c03 = cot(m0, e3), c04 = cot(m0, e4);
      cross3(e0, e1, n1);
      cross3(e0, e2, n2);
      const double A = 0.5 * (std::sqrt(dot3(n1, n1)) + std::sqrt(dot3(n2, n2)));
      const double K[5] = {c03 + c04, c01 + c02, -c01 - c03, -c02 - c04, 3.0 / A};
      NCPADJ_REQUIRE(std::isfinite(K[0] + K[1] + K[2] + K[3] + K[4]), "a degenerate triangle at a bending hinge");
      const int32_t ids[4] = {i0, i1, i2, i3};
      P.bidx.insert(P.bidx.end(), ids, ids + 4);
      P.bcoef.insert(P.bcoef.end(), K, K + 5);
    }
    i = j;
  }
}

static void build_part(const MeshSpec& d, double h, MeshPart& P) {
  const int nv = d.nv, nt = d.ne, k = d.nvpe, gd = k - 1;  // g_a has k - 1 components
  const std::string en = k == 4 ? "tet " : "triangle ";
  NCPADJ_REQUIRE(nv > 0 && nt > 0, "n_verts and the element count must be positive");
  NCPADJ_REQUIRE(d.rest_pos && d.elems && d.E && d.nu, "scene arrays must not be NULL");
  NCPADJ_REQUIRE(d.density > 0 && d.h > 0 && std::isfinite(d.density) && std::isfinite(d.h),
                 "density and h must be positive");
  NCPADJ_REQUIRE(d.h == h, "every scene of a batch must use the same step size h");
  if (k == 3)
    NCPADJ_REQUIRE(d.thickness > 0 && std::isfinite(d.thickness) && d.bend >= 0 && std::isfinite(d.bend),
                   "a shell needs thickness > 0 and bend >= 0");
  P.gvec.assign((size_t)k * gd * nt, 0.0);
  P.vol.assign(nt, 0.0);
  P.mu.assign(nt, 0.0);
  P.lam.assign(nt, 0.0);
  P.lame_d.assign(4 * (size_t)nt, 0.0);
  P.mass.assign(nv, 0.0);
  for (int t = 0; t < nt; ++t) {
    int v[4];
    for (int a = 0; a < k; ++a) {
      v[a] = d.elems[(size_t)k * t + a];
      NCPADJ_REQUIRE(v[a] >= 0 && v[a] < nv, en + std::to_string(t) + " has a vertex index out of range");
    }
    double* g = P.gvec.data() + (size_t)k * gd * t;
    P.vol[t] = k == 4 ? tet_rest(d.rest_pos, v, t, g) : d.thickness * tri_rest(d.rest_pos, v, t, g);
    const double E = d.E[t], nu = d.nu[t];
    NCPADJ_REQUIRE(E > 0 && nu > -1.0 && nu < 0.5 && std::isfinite(E),
                   en + std::to_string(t) + ": need E > 0 and -1 < nu < 0.5");
    P.mu[t] = E / (2.0 * (1.0 + nu));
    P.lam[t] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    P.lame_d[4 * t + 0] = 1.0 / (2.0 * (1.0 + nu));
    P.lame_d[4 * t + 1] = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    P.lame_d[4 * t + 2] = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
    const double q = (1.0 + nu) * (1.0 - 2.0 * nu);
    P.lame_d[4 * t + 3] = E * (1.0 + 2.0 * nu * nu) / (q * q);
    for (int a = 0; a < k; ++a) P.mass[v[a]] += d.density * P.vol[t] / k;
  }
  P.bidx.clear();
  P.bcoef.clear();
  if (k == 3) bending_hinges(d, P);
  const int nh = (int)P.bidx.size() / 4;
  // block pattern: vertices sharing an element or a hinge (sorted neighbour lists, self included)
  std::vector<std::vector<int32_t>> nbr(nv);
  for (int v = 0; v < nv; ++v) nbr[v].push_back(v);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) nbr[d.elems[(size_t)k * t + a]].push_back(d.elems[(size_t)k * t + b]);
  for (int e = 0; e < nh; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) nbr[P.bidx[4 * e + a]].push_back(P.bidx[4 * e + b]);
  P.row_ptr.assign(nv + 1, 0);
  P.col.clear();
  for (int v = 0; v < nv; ++v) {
    auto& L = nbr[v];
    std::sort(L.begin(), L.end());
    L.erase(std::unique(L.begin(), L.end()), L.end());
    P.row_ptr[v + 1] = P.row_ptr[v] + (int)L.size();
    P.col.insert(P.col.end(), L.begin(), L.end());
  }
  auto find_slot = [&](int u, int w) {
    auto b = P.col.begin() + P.row_ptr[u], e = P.col.begin() + P.row_ptr[u + 1];
    return (int32_t)(std::lower_bound(b, e, w) - P.col.begin());
  };
  P.slot.assign((size_t)k * k * nt, 0);
  P.diag_slot.assign(nv, 0);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b)
        P.slot[(size_t)k * k * t + k * a + b] = find_slot(d.elems[(size_t)k * t + a], d.elems[(size_t)k * t + b]);
  for (int v = 0; v < nv; ++v) P.diag_slot[v] = find_slot(v, v);
  P.bslot.assign(16 * (size_t)nh, 0);
  for (int e = 0; e < nh; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) P.bslot[16 * e + 4 * a + b] = find_slot(P.bidx[4 * e + a], P.bidx[4 * e + b]);
  // scalar elastic matrix A_s = M_s + h^2 sum_i w_i (g_a . g_b) + h^2 bend Q_s, w_i = 2 mu_i V_i
  CsrD As;
  As.n = nv;
  As.ptr.assign(P.row_ptr.begin(), P.row_ptr.end());
  As.col = P.col;
  As.val.assign(P.col.size(), 0.0);
  for (int v = 0; v < nv; ++v) As.val[P.diag_slot[v]] += P.mass[v];
  const double h2 = d.h * d.h;
  for (int t = 0; t < nt; ++t) {
    const double w = 2.0 * P.mu[t] * P.vol[t];
    const double* g = P.gvec.data() + (size_t)k * gd * t;
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        double gg = 0;
        for (int c = 0; c < gd; ++c) gg += g[gd * a + c] * g[gd * b + c];
        As.val[P.slot[(size_t)k * k * t + k * a + b]] += h2 * w * gg;
      }
  }
  for (int e = 0; e < nh; ++e) {
    const double* K = P.bcoef.data() + 5 * (size_t)e;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) As.val[P.bslot[16 * e + 4 * a + b]] += h2 * d.bend * K[4] * K[a] * K[b];
  }
  auto t0 = std::chrono::steady_clock::now();
  factor_elastic(As, d.rest_pos, P.F);
  P.ms_factor = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// A scene is the disjoint union of one or more meshes (a batch): vertex and tet ids of mesh s are
// offset by the counts of meshes 0..s-1.  Each mesh's factor is computed independently (in
// parallel) and the union's matrices are block-diagonal.
static void build_scene(Scene& S, const MeshSpec* descs, int n_scenes) {
  NCPADJ_REQUIRE(n_scenes >= 1 && descs, "need at least one scene description");
  const double h = descs[0].h;
  const int nvpe = descs[0].nvpe;
  for (int i = 0; i < n_scenes; ++i)
    NCPADJ_REQUIRE(descs[i].nvpe == nvpe, "a batch mixes tet meshes and shells");
  std::vector<MeshPart> parts(n_scenes);
  std::vector<Error> errs(n_scenes, Error{NCPADJ_OK, ""});
  {
    const int nth = std::max(1, std::min<int>(n_scenes, (int)std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    for (int w = 0; w < nth; ++w)
      pool.emplace_back([&]() {
        for (int i = next++; i < n_scenes; i = next++) {
          try {
            build_part(descs[i], h, parts[i]);
          } catch (const Error& e) {
            errs[i] = e;
          } catch (const std::exception& e) {
            errs[i] = Error{NCPADJ_ERR_OOM, e.what()};
          }
        }
      });
    for (auto& t : pool) t.join();
  }
  for (int i = 0; i < n_scenes; ++i)
    if (errs[i].status != NCPADJ_OK)
      throw Error{errs[i].status, (n_scenes > 1 ? "scene " + std::to_string(i) + ": " : std::string()) + errs[i].msg};
  // union with offsets
  S.n_scenes = n_scenes;
  S.voff.assign(n_scenes + 1, 0);
  S.toff.assign(n_scenes + 1, 0);
  for (int i = 0; i < n_scenes; ++i) {
    S.voff[i + 1] = S.voff[i] + descs[i].nv;
    S.toff[i + 1] = S.toff[i] + descs[i].ne;
  }
  const int nv = S.voff[n_scenes], nt = S.toff[n_scenes];
  S.nv = nv;
  S.nt = nt;
  S.h = h;
  S.density = descs[0].density;
  S.nvpe = nvpe;
  std::vector<double> gvec, vol, mu, lam, lame_d, bcoef, bkb;
  std::vector<int32_t> tets, row_ptr(1, 0), col, slot, diag_slot, perm, iperm, scene_of_vertex, bidx, bslot,
      beoff(1, 0);
  S.mass.clear();
  CsrD Su, Stu;  // union sparse inverse (position space of the union = concatenated positions)
  Su.n = Stu.n = nv;
  Su.ptr.assign(1, 0);
  Stu.ptr.assign(1, 0);
  int64_t nnz_L = 0;
  double ms = 0;
  for (int i = 0; i < n_scenes; ++i) {
    const MeshPart& P = parts[i];
    const int vo = S.voff[i];
    const int bo = (int)col.size();
    gvec.insert(gvec.end(), P.gvec.begin(), P.gvec.end());
    vol.insert(vol.end(), P.vol.begin(), P.vol.end());
    mu.insert(mu.end(), P.mu.begin(), P.mu.end());
    lam.insert(lam.end(), P.lam.begin(), P.lam.end());
    lame_d.insert(lame_d.end(), P.lame_d.begin(), P.lame_d.end());
    S.mass.insert(S.mass.end(), P.mass.begin(), P.mass.end());
    for (size_t t = 0; t < (size_t)descs[i].ne * nvpe; ++t) tets.push_back(descs[i].elems[t] + vo);
    for (int v = 0; v < descs[i].nv; ++v) row_ptr.push_back(bo + P.row_ptr[v + 1]);
    for (int32_t x : P.bidx) bidx.push_back(x + vo);
    for (int32_t x : P.bslot) bslot.push_back(x + bo);
    bcoef.insert(bcoef.end(), P.bcoef.begin(), P.bcoef.end());
    bkb.insert(bkb.end(), P.bidx.size() / 4, descs[i].bend);
    beoff.push_back(beoff.back() + (int32_t)(P.bidx.size() / 4));
    for (int32_t c : P.col) col.push_back(c + vo);
    for (int32_t x : P.slot) slot.push_back(x + bo);
    for (int32_t x : P.diag_slot) diag_slot.push_back(x + bo);
    for (int32_t x : P.F.perm) perm.push_back(x + vo);
    for (int32_t x : P.F.iperm) iperm.push_back(x + vo);
    scene_of_vertex.insert(scene_of_vertex.end(), descs[i].nv, i);
    const int64_t so = (int64_t)Su.col.size(), sto = (int64_t)Stu.col.size();
    for (int r = 0; r < P.F.n; ++r) {
      Su.ptr.push_back(so + P.F.S.ptr[r + 1]);
      Stu.ptr.push_back(sto + P.F.St.ptr[r + 1]);
    }
    for (int32_t c : P.F.S.col) Su.col.push_back(c + vo);  // position space (x is permuted first)
    Su.val.insert(Su.val.end(), P.F.S.val.begin(), P.F.S.val.end());
    for (int32_t c : P.F.St.col) Stu.col.push_back(c + vo);  // position space
    Stu.val.insert(Stu.val.end(), P.F.St.val.begin(), P.F.St.val.end());
    nnz_L += P.F.nnz_L;
    ms += P.ms_factor;
  }
  S.nb = (int)col.size();
  S.ms_factor = ms;
  S.nnz_L = nnz_L;
  S.nnz_S = (int64_t)Su.col.size();
  upload(S.tets, tets);
  upload(S.gvec, gvec);
  upload(S.vol, vol);
  upload(S.mu, mu);
  upload(S.lam, lam);
  upload(S.lame_d, lame_d);
  upload(S.massd, S.mass);
  upload(S.row_ptr, row_ptr);
  upload(S.col, col);
  upload(S.slot, slot);
  upload(S.diag_slot, diag_slot);
  upload(S.perm, perm);
  upload(S.iperm, iperm);
  upload(S.scene_of_vertex, scene_of_vertex);
  S.n_bend = beoff.back();
  upload(S.bend_idx, bidx);
  upload(S.bend_coef, bcoef);
  upload(S.bend_kb, bkb);
  upload(S.bend_slot, bslot);
  upload(S.bend_eoff, beoff);
  upload(S.S_ptr, Su.ptr);
  upload(S.S_val, Su.val);
  upload(S.St_ptr, Stu.ptr);
  upload(S.St_col, Stu.col);
  upload(S.St_val, Stu.val);
  {
    std::vector<float> f1(Su.val.begin(), Su.val.end()), f2(Stu.val.begin(), Stu.val.end());
    upload(S.S_val32, f1);
    upload(S.St_val32, f2);
  }
  S.St_ptr_h = Stu.ptr;
  {  // rows of S are contiguous column ranges (postordered factor): a chunk needs only its first column
    S.S_ptr_h = Su.ptr;
    S.S_first_h.assign(Su.n, 0);
    for (int i = 0; i < Su.n; ++i) {
      const int64_t p0 = Su.ptr[i], p1 = Su.ptr[i + 1];
      if (p1 > p0) S.S_first_h[i] = Su.col[p0];
      for (int64_t q = p0; q < p1; ++q)
        if (Su.col[q] != Su.col[p0] + (int32_t)(q - p0))
          throw Error{NCPADJ_ERR_NOT_FACTORED, "internal: a row of the sparse inverse is not a column range"};
    }
  }
  rechunk(S, S.chunk);
  // host-side resources, made once per scene (a refactor rebuilds only the arrays above)
  S.flags.ensure(FLAG_COUNT * sizeof(int));
  if (!S.flags_host) NCPADJ_CUDA_TRY(cudaMallocHost(&S.flags_host, FLAG_COUNT * sizeof(int)));
  if (!S.scal_host) NCPADJ_CUDA_TRY(cudaMallocHost(&S.scal_host, 16 * sizeof(double)));
  if (!S.gs_host) NCPADJ_CUDA_TRY(cudaMallocHost(&S.gs_host, 2 * (2 * 513 + 1) * sizeof(double)));  // two slots
  for (auto& e : S.gs_ev)
    if (!e) NCPADJ_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  if (!S.gs_inner_host) NCPADJ_CUDA_TRY(cudaMallocHost(&S.gs_inner_host, 256 * sizeof(double)));
  if (!S.gs_map_host) {
    NCPADJ_CUDA_TRY(cudaHostAlloc(&S.gs_map_host, 2 * (2 * 513 + 1) * sizeof(double), cudaHostAllocMapped));
    NCPADJ_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&S.gs_map_dev), S.gs_map_host, 0));
  }
  S.gstep.ensure(64);
  for (auto& e : S.ev)
    if (!e) NCPADJ_CUDA_TRY(cudaEventCreate(&e));
  // tiles of the DOF range that never straddle two meshes (per-scene reductions of a batch solve)
  {
    std::vector<int32_t> tsc, tb, te, t0(n_scenes + 1, 0);
    for (int i = 0; i < n_scenes; ++i) {
      for (int b = 3 * S.voff[i]; b < 3 * S.voff[i + 1]; b += kSegTile) {
        tsc.push_back(i);
        tb.push_back(b);
        te.push_back(std::min(b + kSegTile, 3 * S.voff[i + 1]));
      }
      t0[i + 1] = (int32_t)tsc.size();
    }
    S.n_tiles = (int)tsc.size();
    std::vector<int32_t> all;
    all.insert(all.end(), tsc.begin(), tsc.end());
    all.insert(all.end(), tb.begin(), tb.end());
    all.insert(all.end(), te.begin(), te.end());
    all.insert(all.end(), t0.begin(), t0.end());
    upload(S.segt, all);
  }
  if (!S.bmap_host) {
    NCPADJ_CUDA_TRY(cudaHostAlloc(&S.bmap_host, sizeof(int) * (kMaxRestart + 8), cudaHostAllocMapped));
    NCPADJ_CUDA_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&S.bmap_dev), S.bmap_host, 0));
  }
  for (auto& e : S.bev)
    if (!e) NCPADJ_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // captured steps read the arrays above: they are captured again on their next use
  if (S.step_exec) cudaGraphExecDestroy(S.step_exec);
  if (S.bstep_exec) cudaGraphExecDestroy(S.bstep_exec);
  S.step_exec = S.bstep_exec = nullptr;
  S.step_key.clear();
  S.bstep_key.clear();
}

// host copies of the meshes a scene was built from, so that it can be refactored with new materials
static void keep_geometry(Scene& S, const MeshSpec* descs, int n_scenes) {
  S.geo_pos.assign(n_scenes, {});
  S.geo_tets.assign(n_scenes, {});
  S.geo_density.assign(n_scenes, 0.0);
  S.geo_thickness.assign(n_scenes, 0.0);
  S.mat_bend.assign(n_scenes, 0.0);
  S.mat_E.clear();
  S.mat_nu.clear();
  for (int i = 0; i < n_scenes; ++i) {
    const MeshSpec& d = descs[i];
    S.geo_pos[i].assign(d.rest_pos, d.rest_pos + 3 * (size_t)d.nv);
    S.geo_tets[i].assign(d.elems, d.elems + (size_t)d.nvpe * d.ne);
    S.geo_density[i] = d.density;
    S.geo_thickness[i] = d.thickness;
    S.mat_bend[i] = d.bend;
    S.mat_E.insert(S.mat_E.end(), d.E, d.E + d.ne);
    S.mat_nu.insert(S.mat_nu.end(), d.nu, d.nu + d.ne);
  }
}

// New Young's moduli and Poisson ratios (host arrays [n_tets] over the whole scene) and bending
// stiffnesses ([n_scenes], shells): every material-dependent array and the elastic factor are
// rebuilt from the kept geometry.
static void refactor_scene(Scene& S, const double* E, const double* nu, const double* bend) {
  const int ns = S.n_scenes;
  const std::vector<double> e(E, E + S.nt), n(nu, nu + S.nt), b(bend, bend + ns);  // may alias S.mat_*
  std::vector<MeshSpec> descs(ns);
  for (int i = 0; i < ns; ++i) {
    MeshSpec& m = descs[i];
    const int t0 = S.toff[i];
    m.nv = S.voff[i + 1] - S.voff[i];
    m.ne = S.toff[i + 1] - S.toff[i];
    m.nvpe = S.nvpe;
    m.rest_pos = S.geo_pos[i].data();
    m.elems = S.geo_tets[i].data();
    m.E = e.data() + t0;
    m.nu = n.data() + t0;
    m.density = S.geo_density[i];
    m.h = S.h;
    m.thickness = S.geo_thickness[i];
    m.bend = b[i];
  }
  build_scene(S, descs.data(), ns);
  S.mat_E = e;
  S.mat_nu = n;
  S.mat_bend = b;
}

// ------------------------------------------------------------------------------------------
// the solve engine shared by the adjoint step and the forward Newton step
// ------------------------------------------------------------------------------------------
namespace {

struct Inputs {  // device pointers for one call
  const int32_t* cvertex = nullptr;
  const double* frame = nullptr;
  const double* d_n = nullptr;
  const double* d_f = nullptr;
  const double* mu = nullptr;
  const int32_t* region = nullptr;
  const double* q = nullptr;
  const double* q_prev = nullptr;
  const double* lambda = nullptr;
  const double* dL_dq = nullptr;
  const double* dL_dv = nullptr;
  int nbind = 0;  // bilateral bindings (device arrays)
  const int32_t* bvertex = nullptr;
  const double* btarget = nullptr;
  const double* bcompliance = nullptr;
  const int32_t* btet = nullptr;  // points inside tets (with bbary [nbind][4]) instead of vertices
  const double* bbary = nullptr;
};

struct Engine {
  Scene& S;
  const Ctx& C;
  cudaStream_t st;
  int nv = 0, nt = 0, nc = 0, N = 0, ncap = 0, m = 64, precond = NCPADJ_PRECOND_WOODBURY, transpose = 1;
  double h = 0;
  Inputs in;
  int* flags = nullptr;
  // vectors [N]
  double *b, *x, *r, *w, *t0, *t1, *t2, *t3, *dinv;
  // contact-space vectors [ncap]
  double *sc, *tc, *ytmp;
  double *partial, *scal;
  double *Ds = nullptr, *Cm = nullptr;
  int32_t* piv = nullptr;
  bool cap_timed = false;
  // mixed precision: FP32 matrix values, FP32 A^{-1} products and capacitance apply
  bool mixed = false;
  bool cap_fp32 = false;  // factorise the capacitance in FP32 as well
  bool cap_tc = false;    // ... by the blocked Gauss-Jordan on the tensor cores (else pivoted Gauss-Jordan)
  int cap_nmax = 0;       // largest capacitance block (rows); S.capmeta holds the block table

  // x = C^{-1} y over every directly inverted capacitance block, in one launch
  void cap_apply_all(const double* y, double* x, const int* act = nullptr) {
    const int nbk = (int)blk_c0.size();
    launch_cap_apply_all(nbk, cap_nmax, S.capmeta.as<int64_t>(), (mixed || cap_fp32) ? Cm32 : nullptr,
                         (mixed || cap_fp32) ? nullptr : Cm, piv, y, x, act, st);
    if (cap_refine) {  // one step of iterative refinement against the FP64 capacitance: x += X (y - C x)
      double* r = S.capres.as<double>();
      launch_cap_resid_all(nbk, cap_nmax, S.capmeta.as<int64_t>(), Cm, y, x, r, act, st);
      launch_cap_apply_all(nbk, cap_nmax, S.capmeta.as<int64_t>(), Cm32, nullptr, piv, r, x, act, st, true);
    }
  }
  bool cap_refine = false;  // NCPADJ_REFINED: FP32 inverse, each solve refined against the FP64 capacitance
  int cap_block = 0;      // most contacts per capacitance block (0: the largest the direct inverse takes)
  float *x32 = nullptr, *w32 = nullptr, *Cm32 = nullptr;
  float2* zsplit = nullptr;  // double-float pairs of the Arnoldi matvec's input (mixed)
  // the capacitance is block-diagonal by scene (contacts of different meshes share no ancestor
  // in the elimination forest): one dense block per scene that has contacts
  // The contacts of the Woodbury capacitance (select_capacitance): every contact except those whose
  // capacitance rows are within cap_drop of the identity; the assembled matrix and the contractions
  // always take every contact.
  int cnc = 0;
  int nbc = 0;                   // single-vertex bindings among the candidates (after the contacts)
  const int32_t* cvx = nullptr;  // [cnc] vertex ids
  const double* cfr = nullptr;   // [cnc][9] frames
  const double* ccd = nullptr;   // [cnc][12] K, k_mu
  double cap_drop = 0.0;
  std::vector<int> blk_c0, blk_nc, blk_scene;  // first contact, contacts and mesh of each block
  std::vector<size_t> blk_moff, blk_doff;
  // batch scenes: one restarted GMRES per mesh, all meshes advanced by the same launches
  bool batch_mode = false;
  struct BatchBufs {
    int ns = 0, K = 0, gstride = 0;
    int *act = nullptr, *cyc = nullptr, *done = nullptr, *kk = nullptr, *iters = nullptr;
    double *gsb = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *bnorm = nullptr, *tol = nullptr, *rr = nullptr, *relres = nullptr, *partial = nullptr;
    unsigned* cnt = nullptr;
  } bb;
  size_t cap_elems = 0, ds_elems = 0;
  // scene blocks above the direct inverse's size are solved iteratively (Sec. 4.4: inner Krylov
  // solve on the capacitance): an inner right-preconditioned GMRES applies the capacitance of such
  // a block without forming it (cap_matvec) and is preconditioned by the exact inverse of each of
  // its contiguous groups (blk_*).  sup_g0/sup_g1: the groups of super-block k.
  std::vector<int> sup_c0, sup_nc, sup_g0, sup_g1;
  static constexpr int kInnerRestart = 40;
  double inner_rtol = 1e-6;
  int inner_iters = 0;

  // the capacitance blocks over the contacts of the capacitance set (cnc of them)
  void plan_blocks() {
    blk_c0.clear();
    blk_nc.clear();
    blk_scene.clear();
    if (cnc == 0) return;
    std::vector<int> bsc;  // mesh of each block
    if (S.n_scenes == 1) {
      blk_c0.push_back(0);
      blk_nc.push_back(cnc);
      bsc.push_back(0);
    } else {
      S.cscene.ensure(sizeof(int32_t) * (size_t)cnc + 64);
      launch_contact_scene(cnc, cvx, S.scene_of_vertex.as<int32_t>(), S.cscene.as<int32_t>(), st);
      std::vector<int32_t> cs(cnc);
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(cs.data(), S.cscene.as<int32_t>(), sizeof(int32_t) * cnc,
                                      cudaMemcpyDeviceToHost, st));
      NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
      for (int c = 0; c < cnc; ++c) {
        NCPADJ_REQUIRE(c == 0 || cs[c] >= cs[c - 1], "contacts of a batch scene must be grouped by scene");
        if (c == 0 || cs[c] != cs[c - 1]) {
          blk_c0.push_back(c);
          blk_nc.push_back(0);
          bsc.push_back(cs[c]);
        }
        blk_nc.back()++;
      }
    }
    // blocks above the direct inverse's size (or the caller's limit) are split into contiguous,
    // nearly equal groups; the Delassus coupling between groups is left out of the preconditioner
    {
      // direct inverse up to 2,730 contacts (8,190 rows) by default: beyond that the inversion, DRAM
      // bound at ~2n^3/BP bytes, costs more than the inner iterations; FP64 stops at 4,096 rows
      const int dmax = (cap_fp32 ? std::min(gj_cols_max_dim(), 8190) : gj_cols_max_dim64()) / 3;
      const int lim = cap_block > 0 ? std::min(cap_block, (cap_fp32 ? gj_cols_max_dim() : gj_cols_max_dim64()) / 3)
                                    : dmax;
      std::vector<int> c0s, ncs;
      sup_c0.clear();
      sup_nc.clear();
      sup_g0.clear();
      sup_g1.clear();
      for (size_t b = 0; b < blk_c0.size(); ++b) {
        const int parts = (blk_nc[b] + lim - 1) / lim;
        if (parts > 1) {
          sup_c0.push_back(blk_c0[b]);
          sup_nc.push_back(blk_nc[b]);
          sup_g0.push_back((int)c0s.size());
          sup_g1.push_back((int)c0s.size() + parts);
        }
        for (int k = 0; k < parts; ++k) {
          const int lo = blk_c0[b] + (int)((long)blk_nc[b] * k / parts);
          const int hi = blk_c0[b] + (int)((long)blk_nc[b] * (k + 1) / parts);
          c0s.push_back(lo);
          ncs.push_back(hi - lo);
          blk_scene.push_back(bsc[b]);
        }
      }
      blk_c0.swap(c0s);
      blk_nc.swap(ncs);
      // the per-scene batch solve runs every step as one captured launch sequence, with no inner
      // solve: the groups of a large block are then inverted directly and their coupling is left
      // out of the preconditioner (flexible GMRES keeps the result exact)
      if (batch_mode) {
        sup_c0.clear();
        sup_nc.clear();
        sup_g0.clear();
        sup_g1.clear();
      }
    }
    blk_moff.assign(blk_c0.size(), 0);
    blk_doff.assign(blk_c0.size(), 0);
    cap_elems = ds_elems = 0;
    for (size_t b = 0; b < blk_c0.size(); ++b) {
      blk_moff[b] = cap_elems;
      blk_doff[b] = ds_elems;
      cap_elems += (size_t)9 * blk_nc[b] * blk_nc[b];
      ds_elems += (size_t)blk_nc[b] * blk_nc[b];
    }
  }
  SinvArgs sinv{};

  Engine(Scene& s, const Ctx& c, cudaStream_t stream) : S(s), C(c), st(stream) {
    nv = S.nv;
    nt = S.nt;
    N = 3 * nv;
    h = S.h;
    flags = S.flags.as<int>();
  }

  // capacitance matrices, the inverse's scratch and the inner solve's basis for the current plan
  void alloc_capacitance() {
    if (mixed || cap_fp32) {
      S.vec32.ensure(sizeof(float) * (2 * (size_t)N + cap_elems + 64));
      x32 = S.vec32.as<float>();
      w32 = x32 + N;
      Cm32 = w32 + N;
    }
    if ((nc + nbc) && precond == NCPADJ_PRECOND_WOODBURY) {
      S.cap.ensure(sizeof(double) * (cap_elems + ds_elems + 16) + sizeof(int32_t) * ((size_t)ncap + 16));
      int nmax = 0;
      for (int v : blk_nc) nmax = std::max(nmax, 3 * v);
      const size_t wbytes = gj_cols_scratch_bytes(nmax, false);
      if (S.capw.bytes < wbytes) {  // the column-owned inverse expects its flags zero
        S.capw.ensure(wbytes);
        NCPADJ_CUDA_TRY(cudaMemset(S.capw.p, 0, wbytes));
      }
      Cm = S.cap.as<double>();
      Ds = Cm + cap_elems;
      if (cap_refine) S.capres.ensure(sizeof(double) * ((size_t)ncap + 16));
      piv = reinterpret_cast<int32_t*>(Ds + ds_elems + 16);
      if (!sup_c0.empty()) {
        int smax = 0;
        for (int v : sup_nc) smax = std::max(smax, 3 * v);
        S.inner.ensure(sizeof(double) * ((size_t)(kInnerRestart + 1) * smax + 3 * (size_t)smax +
                                         2 * (size_t)(kInnerRestart + 2) + 64));
      }
    }
  }

  void workspace(int nc_, int m_, int precond_) {
    nc = nc_;
    m = m_;
    precond = precond_;
    // single-vertex bindings join the capacitance (one scene: a batch groups it by mesh)
    nbc = (S.n_scenes == 1 && in.nbind > 0 && in.bvertex && precond_ == NCPADJ_PRECOND_WOODBURY) ? in.nbind : 0;
    ncap = 3 * (nc + nbc);
    S.cdata.ensure(sizeof(double) * 12 * (size_t)std::max(nc, 1));
    cnc = nc + nbc;  // until select_capacitance: every candidate (the largest plan)
    cvx = in.cvertex;
    cfr = in.frame;
    ccd = S.cdata.as<double>();
    plan_blocks();
    if (mixed) S.bsr32.ensure(sizeof(float) * 9 * (size_t)S.nb);
    else S.bsr64.ensure(sizeof(double) * 9 * (size_t)S.nb);
    if (mixed) {
      S.xsplit.ensure(sizeof(float2) * (size_t)N + 64);
      zsplit = S.xsplit.as<float2>();
    }
    S.tetdata.ensure(sizeof(double) * 18 * (size_t)nt);
    const size_t nvec = 9, ncv = 3 * (size_t)std::max(ncap, 1);
    S.vecs.ensure(sizeof(double) * (nvec * N + ncv + 64));
    // (m + 1) basis vectors and the coefficient slots; at least 7 vectors (BiCGSTAB's)
    S.gmres.ensure(sizeof(double) * ((size_t)std::max(m + 1, 7) * N + 3 * (size_t)(m + 1) + 16));
    if (S.red.bytes < dot_scratch_bytes()) {  // counters of the fused dot product start at zero
      S.red.ensure(dot_scratch_bytes());
      NCPADJ_CUDA_TRY(cudaMemset(S.red.p, 0, dot_scratch_bytes()));
    }
    S.scal.ensure(sizeof(double) * (64 + (size_t)m + 8));
    alloc_capacitance();
    if (flexible_gmres() || batch_mode) S.fgmres.ensure(sizeof(double) * (size_t)(m + 1) * N);
    if (batch_mode) {
      const int ns = S.n_scenes;
      bb.ns = ns;
      bb.K = m + 3;
      bb.gstride = 2 * (m + 1) + 1;
      const size_t nd = (size_t)ns * bb.gstride + (size_t)ns * (m + 1) * m + 2 * (size_t)ns * m +
                        (size_t)ns * (m + 1) + (size_t)ns * m + 4 * (size_t)ns + (size_t)(m + 1) * S.n_tiles;
      const size_t ni = 5 * (size_t)ns + (size_t)ns * bb.K;
      S.bwork.ensure(sizeof(double) * nd + sizeof(int) * ni + 256);
      double* d = S.bwork.as<double>();
      auto take = [&](size_t n) {
        double* r = d;
        d += n;
        return r;
      };
      bb.gsb = take((size_t)ns * bb.gstride);
      bb.H = take((size_t)ns * (m + 1) * m);
      bb.cs = take((size_t)ns * m);
      bb.sn = take((size_t)ns * m);
      bb.g = take((size_t)ns * (m + 1));
      bb.y = take((size_t)ns * m);
      bb.bnorm = take(ns);
      bb.tol = take(ns);
      bb.rr = take(ns);
      bb.relres = take(ns);
      bb.partial = take((size_t)(m + 1) * S.n_tiles);
      int* ip = reinterpret_cast<int*>(d);
      bb.act = ip;
      bb.cyc = ip + ns;
      bb.done = ip + 2 * ns;
      bb.kk = ip + 3 * ns;
      bb.iters = ip + 4 * ns;
      bb.cnt = reinterpret_cast<unsigned*>(ip + 5 * ns);
    }
    double* base = S.vecs.as<double>();
    for (double** v : {&b, &x, &r, &w, &t0, &t1, &t2, &t3, &dinv}) {
      *v = base;
      base += N;
    }
    const size_t nv3 = std::max(ncap, 1);
    sc = base; base += nv3;
    tc = base; base += nv3;
    ytmp = base; base += nv3;
    partial = S.red.as<double>();
    scal = S.scal.as<double>();
    sinv = SinvArgs{nv, S.S_ptr.as<int64_t>(), S.S_c0.as<int32_t>(), S.S_val.as<double>(), S.St_ptr.as<int64_t>(),
                    S.St_col.as<int32_t>(), S.St_val.as<double>(), S.perm.as<int32_t>(), S.nS_chunks, S.nSt_chunks,
                    S.S_crow.as<int32_t>(), S.St_crow.as<int32_t>(), S.S_cbeg.as<int64_t>(), S.S_cend.as<int64_t>(),
                    S.St_cbeg.as<int64_t>(), S.St_cend.as<int64_t>(), S.S_val32.as<float>(), S.St_val32.as<float>()};
    sinv.chunk = S.chunk;
    S.xpos.ensure(sizeof(double) * N + sizeof(float) * N + 64);
    sinv.xpos = S.xpos.as<double>();
    sinv.xpos32 = reinterpret_cast<float*>(S.xpos.as<double>() + N);
  }

  ContactArgs contact_args(const double* q, const double* q_prev, const double* lambda, double eps) const {
    return ContactArgs{nc, in.cvertex, in.frame, in.d_n, in.d_f, in.mu, lambda, q, q_prev, S.diag_slot.as<int32_t>(),
                       eps, h, transpose, mixed ? nullptr : S.bsr64.as<double>(), mixed ? S.bsr32.as<float>() : nullptr,
                       S.cdata.as<double>(), flags};
  }

  // script_A (transpose = 0) or script_A^T (transpose = 1) at (q, lambda) into the block pattern
  void assemble(const double* q, const double* q_prev, const double* lambda, double eps) {
    double* b64 = mixed ? nullptr : S.bsr64.as<double>();
    float* b32 = mixed ? S.bsr32.as<float>() : nullptr;
    launch_bsr_init(nv, S.nb, S.diag_slot.as<int32_t>(), S.massd.as<double>(), b64, b32, st);
    TetArgs ta{nt, S.tets.as<int32_t>(), S.gvec.as<double>(), S.vol.as<double>(), S.mu.as<double>(), S.lam.as<double>(),
               S.slot.as<int32_t>(), q, h, b64, b32, S.tetdata.as<double>(), flags, S.model_ptr()};
    if (S.nvpe == 3) {
      if (mixed) launch_tri_assemble32(ta, st);
      else launch_tri_assemble64(ta, st);
      launch_bend_blocks(S.n_bend, S.bend_idx.as<int32_t>(), S.bend_coef.as<double>(), S.bend_kb.as<double>(),
                         S.bend_slot.as<int32_t>(), h, b64, b32, st);
    } else if (mixed) {
      launch_tet_assemble32(ta, st);
    } else {
      launch_tet_assemble64(ta, st);
    }
    if (nc) launch_contact_blocks(contact_args(q, q_prev, lambda, eps), st);
    if (in.nbind && in.btet)
      launch_binding_blocks_bary(in.nbind, in.btet, in.bbary, in.bcompliance, S.slot.as<int32_t>(), h, b64, b32, st);
    else if (in.nbind)
      launch_binding_blocks(in.nbind, in.bvertex, in.bcompliance, S.diag_slot.as<int32_t>(), h, b64, b32, st);
    NCPADJ_CUDA_TRY(cudaGetLastError());
  }

  // The capacitance set: contact c stays out when h^2 |K_c|_F (A_s^{-1})_{v_c v_c} <= cap_drop, i.e.
  // when its rows of I + h^2 K^T D stand within about cap_drop of the identity (a separating
  // contact: K_c ~ eps^2 / delta_n^2).  The preconditioner is then the exact Woodbury inverse of
  // A + h^2 J_k^T K_k J_k over the kept contacts; the left-out ones stay in the matrix, and the
  // Krylov solve absorbs them (flexible GMRES: the result keeps its tolerance).
  // Candidates are the contacts followed by the single-vertex bindings (J_b = e_v^T (x) I_3, K = I / E_b,
  // Sec. 3.2.1 puts J_b in the same low-rank term), so that stiff bindings are preconditioned exactly.
  void select_capacitance() {
    const int ncand = nc + nbc;
    cnc = ncand;
    cvx = in.cvertex;
    cfr = in.frame;
    ccd = S.cdata.as<double>();
    if (ncand == 0 || (!(cap_drop > 0.0) && nbc == 0)) return;
    // layout: candidates (vertex, frame, K) when bindings join, then the kept set, scores, indices
    S.capsel.ensure(sizeof(double) * (size_t)ncand * (21 + 21 + 1) + sizeof(int32_t) * 3 * (size_t)ncand + 256);
    double* cand_f = S.capsel.as<double>();
    double* cand_c = cand_f + 9 * (size_t)ncand;
    double* fr = cand_c + 12 * (size_t)ncand;
    double* cd = fr + 9 * (size_t)ncand;
    double* score = cd + 12 * (size_t)ncand;
    int32_t* cand_v = reinterpret_cast<int32_t*>(score + ncand);
    int32_t* idx = cand_v + ncand;
    int32_t* vx = idx + ncand;
    const int32_t* sv = in.cvertex;
    const double* sf = in.frame;
    const double* sd = S.cdata.as<double>();
    if (nbc) {
      if (nc) {
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(cand_v, in.cvertex, sizeof(int32_t) * nc, cudaMemcpyDeviceToDevice, st));
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(cand_f, in.frame, sizeof(double) * 9 * nc, cudaMemcpyDeviceToDevice, st));
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(cand_c, S.cdata.as<double>(), sizeof(double) * 12 * nc,
                                        cudaMemcpyDeviceToDevice, st));
      }
      launch_binding_capdata(nbc, in.bvertex, in.bcompliance, nc, cand_v, cand_f, cand_c, st);
      sv = cand_v;
      sf = cand_f;
      sd = cand_c;
      cvx = sv;
      cfr = sf;
      ccd = sd;
    }
    if (!(cap_drop > 0.0)) return;
    launch_contact_score(ncand, sv, S.iperm.as<int32_t>(), S.St_ptr.as<int64_t>(), S.St_val.as<double>(), sd, h,
                         score, st);
    std::vector<double> sh(ncand);
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(sh.data(), score, sizeof(double) * ncand, cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int32_t> keep;
    keep.reserve(ncand);
    for (int c = 0; c < ncand; ++c)
      if (!(sh[c] <= cap_drop)) keep.push_back(c);  // NaN scores stay in
    if ((int)keep.size() == ncand) return;
    cnc = (int)keep.size();
    if (cnc) {
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(idx, keep.data(), sizeof(int32_t) * cnc, cudaMemcpyHostToDevice, st));
      launch_gather_contacts(cnc, idx, sv, sf, sd, vx, fr, cd, st);
    }
    cvx = vx;
    cfr = fr;
    ccd = cd;
  }

  // The tensor-core inverse pivots only inside its 64 x 64 diagonal blocks; where that meets a nearly
  // singular block its result is no preconditioner.  One probe per capacitance block, y = 1:
  // x = X y, r = y - C x (FP64 C); a block with ||r|| > 0.5 ||y|| is inverted again by the pivoted
  // Gauss-Jordan of gj.cu (blocks of at most smax rows were inverted with full pivoting already).
  void check_tc_inverses(int smax) {
    const int nbk = (int)blk_c0.size();
    S.capchk.ensure(sizeof(double) * 3 * ((size_t)ncap + 16));
    double* yv = S.capchk.as<double>();
    double* xv = yv + ncap + 16;
    double* rv = xv + ncap + 16;
    launch_fill(ncap, 1.0, yv, st);
    launch_cap_apply_all(nbk, cap_nmax, S.capmeta.as<int64_t>(), Cm32, nullptr, piv, yv, xv, nullptr, st);
    launch_cap_resid_all(nbk, cap_nmax, S.capmeta.as<int64_t>(), Cm, yv, xv, rv, nullptr, st);
    std::vector<double> rh((size_t)ncap);
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(rh.data(), rv, sizeof(double) * ncap, cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    cap_fallbacks = 0;
    for (int k = 0; k < nbk; ++k) {
      const int n_ = 3 * blk_nc[k];
      if (n_ <= smax) continue;
      double r2 = 0.0;
      for (int i = 0; i < n_; ++i) r2 += rh[3 * (size_t)blk_c0[k] + i] * rh[3 * (size_t)blk_c0[k] + i];
      if (std::isfinite(r2) && r2 <= 0.25 * n_) continue;
      launch_convert_f32((long)n_ * n_, Cm + blk_moff[k], Cm32 + blk_moff[k], st);
      if (!launch_gj_cols32(n_, Cm32 + blk_moff[k], S.capw.p, piv + 3 * (size_t)blk_c0[k], flags, C.sm_count, st)) {
        cudaGetLastError();
        throw Error{NCPADJ_ERR_UNSUPPORTED,
                    "capacitance block of dimension " + std::to_string(n_) + " does not fit the direct inverse"};
      }
      NCPADJ_CUDA_TRY(cudaGetLastError());
      ++cap_fallbacks;
    }
  }
  int cap_fallbacks = 0;  // blocks the check sent back to the pivoted Gauss-Jordan (last set-up)

  void setup_precond() {
    if (precond == NCPADJ_PRECOND_JACOBI)
      launch_diag_inv(nv, S.diag_slot.as<int32_t>(), mixed ? nullptr : S.bsr64.as<double>(),
                      mixed ? S.bsr32.as<float>() : nullptr, dinv, st);
    if (precond == NCPADJ_PRECOND_WOODBURY && (nc + nbc)) {
      select_capacitance();
      plan_blocks();
      alloc_capacitance();
      {  // block table of the one-launch capacitance apply: element offset, row offset, dimension, scene
        const size_t nbk = blk_c0.size();
        std::vector<int64_t> meta(5 * nbk);
        cap_nmax = 0;
        for (size_t k = 0; k < nbk; ++k) {
          meta[k] = (int64_t)blk_moff[k];
          meta[nbk + k] = 3 * (int64_t)blk_c0[k];
          meta[2 * nbk + k] = 3 * (int64_t)blk_nc[k];
          meta[3 * nbk + k] = k < blk_scene.size() ? blk_scene[k] : 0;
          meta[4 * nbk + k] = (int64_t)blk_doff[k];
          cap_nmax = std::max(cap_nmax, 3 * blk_nc[k]);
        }
        S.capmeta.ensure(sizeof(int64_t) * std::max<size_t>(meta.size(), 4));
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.capmeta.p, meta.data(), sizeof(int64_t) * meta.size(),
                                        cudaMemcpyHostToDevice, st));
        NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));  // meta is a local
      }
      if (cap_tc) {  // its own scratch, sized once for the largest block (capw's sync words must stay zero)
        int nmax = 0;
        for (int v : blk_nc) nmax = std::max(nmax, 3 * v);
        S.recw.ensure(bgj_scratch_bytes(nmax));
      }
      // the capacitance of every block (Delassus, then C = I + h^2 K'^T D), FP32 copies where it is
      // inverted in FP32
      launch_cap_form_all((int)blk_c0.size(), cap_nmax / 3, S.capmeta.as<int64_t>(), cvx, S.iperm.as<int32_t>(),
                          S.St_ptr.as<int64_t>(), S.St_col.as<int32_t>(), S.St_val.as<double>(), Ds, cfr, ccd, h,
                          transpose, Cm, cap_fp32 ? Cm32 : nullptr, st);
      NCPADJ_CUDA_TRY(cudaGetLastError());
      NCPADJ_CUDA_TRY(cudaEventRecord(S.ev[6], st));
      // the inverses: every small block in one launch, one CTA each; the others one by one
      const int smax = small_inverse_max(cap_fp32);
      std::vector<int32_t> small;
      for (size_t k = 0; k < blk_c0.size(); ++k)
        if (3 * blk_nc[k] <= smax) small.push_back((int32_t)k);
      if (!small.empty()) {
        int nmax_small = 0;
        for (int32_t k : small) nmax_small = std::max(nmax_small, 3 * blk_nc[k]);
        S.capids.ensure(sizeof(int32_t) * small.size());
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.capids.p, small.data(), sizeof(int32_t) * small.size(),
                                        cudaMemcpyHostToDevice, st));
        launch_small_inverse((int)small.size(), S.capids.as<int32_t>(), (int)blk_c0.size(), S.capmeta.as<int64_t>(),
                             nmax_small, cap_fp32 ? Cm32 : nullptr, cap_fp32 ? nullptr : Cm, piv, flags, st);
        NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));  // small is a local
      }
      for (size_t k = 0; k < blk_c0.size(); ++k) {
        const int c0 = blk_c0[k], n_ = 3 * blk_nc[k];
        if (n_ <= smax) continue;
        double* Cb = Cm + blk_moff[k];
        int32_t* pb = piv + 3 * c0;
        bool ok;
        if (cap_tc) {
          ok = launch_bgj_inverse(n_, Cm32 + blk_moff[k], n_, S.recw.p, pb, flags, C.sm_count, st);
        } else if (cap_fp32) {
          ok = launch_gj_cols32(n_, Cm32 + blk_moff[k], S.capw.p, pb, flags, C.sm_count, st);
        } else {
          ok = launch_gj_cols64(n_, Cb, S.capw.p, pb, flags, C.sm_count, st);
        }
        if (!ok) {
          cudaGetLastError();
          throw Error{NCPADJ_ERR_UNSUPPORTED,
                      "capacitance block of dimension " + std::to_string(n_) + " does not fit the direct inverse"};
        }
        NCPADJ_CUDA_TRY(cudaGetLastError());
      }
      if (cap_tc) check_tc_inverses(smax);
      NCPADJ_CUDA_TRY(cudaEventRecord(S.ev[7], st));
      cap_timed = true;
      if (!cap_fp32 && mixed) launch_convert_f32((long)cap_elems, Cm, Cm32, st);  // FP64 inverses, FP32 apply
      NCPADJ_CUDA_TRY(cudaGetLastError());
    }
  }

  // out = C y for the contacts of super-block k, without forming C:
  //   C y = y + h^2 K'_c F_c (A^{-1} J^T y)_{v_c},
  // where A^{-1} J^T y at the contact vertices is a scatter of y along the contacts'
  // elimination-tree paths into S P J^T y followed by a gather along the same paths.
  void cap_matvec(size_t k, const double* yseg, double* out_seg) {
    const int c0 = sup_c0[k], m_ = sup_nc[k];
    const int32_t* ip = S.iperm.as<int32_t>();
    double* w64 = mixed ? nullptr : t2;
    float* wf = mixed ? x32 : nullptr;
    if (mixed) NCPADJ_CUDA_TRY(cudaMemsetAsync(wf, 0, sizeof(float) * N, st));
    else NCPADJ_CUDA_TRY(cudaMemsetAsync(w64, 0, sizeof(double) * N, st));
    launch_path_scatter(m_, cvx + c0, ip, sinv, cfr + 9 * (size_t)c0, yseg, 1.0, w64, wf, st);
    launch_path_gather(m_, cvx + c0, ip, sinv, w64, wf, cfr + 9 * (size_t)c0, ccd + 12 * (size_t)c0, transpose,
                       out_seg, st);
    launch_axpby(3 * m_, 1.0, yseg, h * h, out_seg, out_seg, st);
  }

  // out = B^{-1} in over the groups g0..g1-1 of a super-block whose first contact is c0 (segment
  // vectors of length 3 * contacts)
  void group_precond(int g0, int g1, int c0, const double* in_seg, double* out_seg) {
    for (int g = g0; g < g1; ++g) {
      const size_t o = 3 * (size_t)(blk_c0[g] - c0);
      const int n_ = 3 * blk_nc[g];
      int32_t* pb = piv + 3 * (size_t)blk_c0[g];
      if (mixed || cap_fp32) launch_gj_apply32(n_, Cm32 + blk_moff[g], pb, in_seg + o, nullptr, out_seg + o, st);
      else launch_gj_apply(n_, Cm + blk_moff[g], pb, in_seg + o, nullptr, out_seg + o, st);
    }
  }

  // Inner solve C y = s on super-block k by right-preconditioned restarted GMRES (classical
  // Gram-Schmidt twice; Hessenberg on the host), to ||s - C y|| <= inner_rtol ||s||.
  void inner_solve(size_t k, const double* sseg, double* yseg) {
    const int n = 3 * sup_nc[k], c0 = sup_c0[k], mi = kInnerRestart;
    double* V = S.inner.as<double>();               // (mi+1) x n
    double* u = V + (size_t)(mi + 1) * n;            // preconditioned vector
    double* rr = u + n;                              // residual
    double* ww = rr + n;                             // C y scratch
    double* gs = ww + n;                             // [0..mi]: pass 1, [mi+1..2mi+1]: pass 2, [2mi+2]: norm
    double* nrm2 = scal + 5;
    NCPADJ_CUDA_TRY(cudaMemsetAsync(yseg, 0, sizeof(double) * n, st));
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(rr, sseg, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    auto norm_host = [&](const double* a) {
      launch_multi_dot(n, 1, a, n, a, partial, scal + 4, st);
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.gs_inner_host + 2 * (mi + 1) + 1, scal + 4, sizeof(double),
                                      cudaMemcpyDeviceToHost, st));
      NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
      return std::sqrt(S.gs_inner_host[2 * (mi + 1) + 1]);
    };
    const double s0 = norm_host(rr);
    if (!(s0 > 0.0) || !std::isfinite(s0)) return;
    const double tol = inner_rtol * s0;
    double beta = s0;
    std::vector<double> H((size_t)(mi + 1) * mi, 0.0), cs(mi), sn(mi), g(mi + 1), yv(mi);
    for (int cycle = 0; cycle < 50; ++cycle) {
      launch_axpby(n, 1.0 / beta, rr, 0.0, nullptr, V, st);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int kk = 0;
      bool done = false;
      for (int j = 0; j < mi; ++j) {
        double* vn = V + (size_t)(j + 1) * n;
        group_precond(sup_g0[k], sup_g1[k], c0, V + (size_t)j * n, u);
        cap_matvec(k, u, vn);
        launch_multi_dot(n, j + 1, V, n, vn, partial, gs, st);
        launch_multi_axpy(n, j + 1, V, n, gs, vn, st);
        launch_multi_dot(n, j + 1, V, n, vn, partial, gs + (mi + 1), st);
        launch_multi_axpy(n, j + 1, V, n, gs + (mi + 1), vn, st);
        launch_multi_dot(n, 1, vn, n, vn, partial, nrm2, st);
        launch_normalize(n, vn, nrm2, vn, gs + 2 * (mi + 1), st);
        // own pinned buffer: the outer GMRES may have a step's coefficients in flight in gs_host
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.gs_inner_host, gs, sizeof(double) * (2 * (mi + 1) + 1),
                                        cudaMemcpyDeviceToHost, st));
        NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
        double* hcol = &H[(size_t)(mi + 1) * j];
        for (int i = 0; i <= j; ++i) hcol[i] = S.gs_inner_host[i] + S.gs_inner_host[mi + 1 + i];
        hcol[j + 1] = S.gs_inner_host[2 * (mi + 1)];
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
          hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
          hcol[i] = t;
        }
        const double rn = std::hypot(hcol[j], hcol[j + 1]);
        cs[j] = rn > 0 ? hcol[j] / rn : 1.0;
        sn[j] = rn > 0 ? hcol[j + 1] / rn : 0.0;
        hcol[j] = rn;
        hcol[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++inner_iters;
        kk = j + 1;
        const double est = std::fabs(g[j + 1]);
        if (!std::isfinite(est) || est <= tol) {
          done = true;
          break;
        }
      }
      for (int i = kk - 1; i >= 0; --i) {
        double t = g[i];
        for (int jj = i + 1; jj < kk; ++jj) t -= H[(size_t)(mi + 1) * jj + i] * yv[jj];
        yv[i] = t / H[(size_t)(mi + 1) * i + i];
      }
      double* ydev = gs + 2 * (mi + 1) + 1;
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(ydev, yv.data(), sizeof(double) * kk, cudaMemcpyHostToDevice, st));
      launch_combine(n, kk, V, n, ydev, ww, st);        // ww = V y
      group_precond(sup_g0[k], sup_g1[k], c0, ww, u);  // u = B^{-1} V y
      launch_axpby(n, 1.0, yseg, 1.0, u, yseg, st);
      cap_matvec(k, yseg, ww);
      launch_axpby(n, 1.0, sseg, -1.0, ww, rr, st);
      beta = norm_host(rr);
      if (done || !std::isfinite(beta) || beta <= tol) break;
    }
  }

  // yout = B xin for the assembled matrix (rows of scenes outside mk skipped); mixed: FP32 values
  // with double-float products and sums (xin split into zsplit first)
  void matvec(const double* xin, double* yout, const Mask& mk = Mask{}) {
    if (mixed) {
      launch_split(N, xin, zsplit, st);
      launch_bsr_spmv_ff(nv, S.row_ptr.as<int32_t>(), S.col.as<int32_t>(), S.bsr32.as<float>(), zsplit, yout, 0,
                         nullptr, st, mk);
    } else {
      launch_bsr_spmv(nv, S.row_ptr.as<int32_t>(), S.col.as<int32_t>(), S.bsr64.as<double>(), xin, yout, st, mk);
    }
  }
  void ainv(const double* xin, double* yout) {
    if (mixed) launch_ainv32(sinv, xin, x32, w32, yout, st);
    else launch_ainv(sinv, xin, t3, yout, st);
  }

  // yout = P^{-1} xin; uses t0..t3 as scratch (yout must be none of them)
  void apply_precond(const double* xin, double* yout) {
    switch (precond) {
      case NCPADJ_PRECOND_NONE:
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(yout, xin, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        break;
      case NCPADJ_PRECOND_JACOBI:
        launch_mul(N, dinv, xin, yout, st);
        break;
      case NCPADJ_PRECOND_ELASTIC:
        ainv(xin, yout);
        break;
      default: {
        // Woodbury (Eq. woodbury_formula without K^{-1}), written as
        //   y = A^{-1} (x - h^2 J^T C^{-1} K' J A^{-1} x),   A^{-1} = P^T S^T S P:
        // w = S P x once; J A^{-1} x needs A^{-1} x at the contact vertices only, i.e. rows of S^T
        // (elimination-tree paths) against w; the correction enters w along the same paths; then
        // y = P^T S^T w.  One full product with S and one with S^T per apply instead of two each.
        if (cnc == 0) {
          ainv(xin, yout);
          break;
        }
        const int32_t* ip = S.iperm.as<int32_t>();
        if (mixed) launch_sinv_half1_32(sinv, xin, w32, st);
        else launch_sinv_half1(sinv, xin, t3, st);
        launch_path_gather(cnc, cvx, ip, sinv, t3, mixed ? w32 : nullptr, cfr, ccd, transpose, sc, st);
        if (sup_c0.empty()) {
          cap_apply_all(sc, tc);
        } else {
          size_t ks = 0;  // super-blocks in contact order
          for (size_t k = 0; k < blk_c0.size();) {
            if (ks < sup_c0.size() && (int)k == sup_g0[ks]) {
              const size_t o = 3 * (size_t)sup_c0[ks];
              inner_solve(ks, sc + o, tc + o);
              k = sup_g1[ks];
              ++ks;
              continue;
            }
            const size_t o = 3 * (size_t)blk_c0[k];
            const int n_ = 3 * blk_nc[k];
            if (mixed || cap_fp32) launch_gj_apply32(n_, Cm32 + blk_moff[k], piv + o, sc + o, ytmp + o, tc + o, st);
            else launch_gj_apply(n_, Cm + blk_moff[k], piv + o, sc + o, ytmp + o, tc + o, st);
            ++k;
          }
        }
        launch_path_scatter(cnc, cvx, ip, sinv, cfr, tc, -h * h, t3, mixed ? w32 : nullptr, st);
        if (mixed) launch_sinv_half2_32(sinv, w32, yout, st);
        else launch_sinv_half2(sinv, t3, yout, st);
      }
    }
  }

  // ---- captured Arnoldi step (Woodbury, direct capacitance blocks) ----
  // One CUDA graph holds a whole GMRES step: preconditioner apply on V_j, matvec into V_{j+1},
  // Gram-Schmidt twice, normalisation, export of the coefficients to host-mapped slot j % 2 and
  // j <- j + 1, with j read on the device.  Replaying it is one launch per step instead of ~16,
  // which matters because the step is otherwise bound by the host's launch rate.
  // flexible GMRES (keep z_j = P^{-1} v_j and update x with Z y, Saad's FGMRES) whenever P^{-1} is
  // not one fixed linear map to FP64 accuracy: an inner iterative capacitance solve makes it vary,
  // and an FP32 application rounds it, so that P^{-1}(V y) is not the combination of the z_j the
  // Arnoldi relation holds for (that mismatch, relative ~1e-7 times the cancellation in V y, can
  // stop a restarted GMRES from converging)
  bool flexible_gmres() const {
    const bool inner = !sup_c0.empty() && precond == NCPADJ_PRECOND_WOODBURY && nc + nbc > 0;
    const bool fp32 = (mixed && (precond == NCPADJ_PRECOND_WOODBURY || precond == NCPADJ_PRECOND_ELASTIC)) ||
                      (cap_fp32 && precond == NCPADJ_PRECOND_WOODBURY && nc + nbc > 0);
    // contacts left out of the capacitance: the preconditioner is not the matrix's inverse even in
    // exact arithmetic, but it is one fixed map, so plain right-preconditioned GMRES stays exact;
    // flexible GMRES is kept for the rounding cases above only
    return inner || fp32;
  }
  bool step_graph_possible() const {
    return precond == NCPADJ_PRECOND_WOODBURY && cnc > 0 && sup_c0.empty();
  }
  std::vector<uintptr_t> step_key() const {
    std::vector<uintptr_t> k = {(uintptr_t)nc, (uintptr_t)m, (uintptr_t)N, (uintptr_t)mixed, (uintptr_t)cap_fp32,
                                (uintptr_t)transpose, (uintptr_t)cvx, (uintptr_t)cfr, (uintptr_t)ccd,
                                (uintptr_t)cnc,
                                (uintptr_t)S.gmres.p, (uintptr_t)S.vecs.p, (uintptr_t)S.red.p, (uintptr_t)S.scal.p,
                                (uintptr_t)S.cap.p, (uintptr_t)S.vec32.p, (uintptr_t)S.cdata.p, (uintptr_t)S.bsr32.p,
                                (uintptr_t)S.bsr64.p, (uintptr_t)S.xpos.p, (uintptr_t)S.gstep.p,
                                (uintptr_t)flexible_gmres(), (uintptr_t)S.fgmres.p,
                                (uintptr_t)S.gs_map_dev, (uintptr_t)blk_c0.size(), (uintptr_t)S.xsplit.p,
                                (uintptr_t)S.capmeta.p, (uintptr_t)cap_nmax, (uintptr_t)cap_refine,
                                (uintptr_t)S.capres.p, (uintptr_t)S.chunk, (uintptr_t)S.nS_chunks,
                                (uintptr_t)S.nSt_chunks, (uintptr_t)S.S_crow.p, (uintptr_t)S.S_cbeg.p,
                                (uintptr_t)S.S_cend.p, (uintptr_t)S.S_c0.p, (uintptr_t)S.St_crow.p,
                                (uintptr_t)S.St_cbeg.p, (uintptr_t)S.St_cend.p};
    for (size_t b = 0; b < blk_c0.size(); ++b) {
      k.push_back((uintptr_t)blk_c0[b]);
      k.push_back((uintptr_t)blk_nc[b]);
    }
    return k;
  }
  void enqueue_step_indexed(double* V, double* gs, double* nrm2, int* jp) {
    const int32_t* ip = S.iperm.as<int32_t>();
    // z = P^{-1} V_j into w (Woodbury, as in apply_precond)
    launch_sinv_half1_idx(sinv, V, N, jp, mixed ? nullptr : t3, mixed ? w32 : nullptr, st);
    launch_path_gather(cnc, cvx, ip, sinv, t3, mixed ? w32 : nullptr, cfr, ccd, transpose, sc, st);
    cap_apply_all(sc, tc);
    launch_path_scatter(cnc, cvx, ip, sinv, cfr, tc, -h * h, t3, mixed ? w32 : nullptr, st);
    if (mixed) launch_sinv_half2_32(sinv, w32, w, st);
    else launch_sinv_half2(sinv, t3, w, st);
    if (flexible_gmres()) launch_copy_idx(N, w, S.fgmres.as<double>(), N, jp, st);  // Z_j = z
    // V_{j+1} = A z (mixed: FP32 values, double-float products and sums)
    if (mixed) {
      launch_split(N, w, zsplit, st);
      launch_bsr_spmv_ff(nv, S.row_ptr.as<int32_t>(), S.col.as<int32_t>(), S.bsr32.as<float>(), zsplit, V, N, jp, st);
    } else {
      launch_bsr_spmv_idx(nv, S.row_ptr.as<int32_t>(), S.col.as<int32_t>(), S.bsr64.as<double>(), nullptr, w, V, N,
                          jp, st);
    }
    launch_multi_dot_idx(N, m, V, N, jp, false, partial, gs, st);
    launch_multi_axpy_idx(N, V, N, jp, gs, V, st);
    launch_multi_dot_idx(N, m, V, N, jp, false, partial, gs + (m + 1), st);
    launch_multi_axpy_idx(N, V, N, jp, gs + (m + 1), V, st);
    launch_multi_dot_idx(N, m, V, N, jp, true, partial, nrm2, st);
    launch_normalize_idx(N, V, N, jp, nrm2, gs + 2 * (m + 1), st);
    launch_export_step(gs, 2 * (m + 1) + 1, S.gs_map_dev, jp, st);
  }
  // the graph for the current configuration (captured on first use and when it changes); null if
  // capture is not possible here
  cudaGraphExec_t step_graph(double* V, double* gs, double* nrm2) {
    if (!step_graph_possible()) return nullptr;
    std::vector<uintptr_t> key = step_key();
    if (S.step_exec && key == S.step_key) return S.step_exec;
    if (S.step_exec) {
      cudaGraphExecDestroy(S.step_exec);
      S.step_exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    const int64_t l0 = g_launches;
    enqueue_step_indexed(V, gs, nrm2, S.gstep.as<int>());
    S.step_launches = (int)(g_launches - l0);
    g_launches = l0;  // counted when the graph is replayed
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (ce != cudaSuccess || !g) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return nullptr;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    S.step_exec = ex;
    S.step_key = key;
    return ex;
  }
  // ---- batched per-scene GMRES (batch scenes) ----
  SegTiles tiles() const {
    const int32_t* t = S.segt.as<int32_t>();
    const int n = S.n_tiles;
    return SegTiles{n, t, t + n, t + 2 * (size_t)n, t + 3 * (size_t)n};
  }
  // One Arnoldi step j = *jp of every active scene (right-preconditioned, flexible: Z_j = P^{-1} V_j
  // is kept).  Every kernel skips the rows of scenes whose act[] is 0; the last one updates each
  // active scene's Hessenberg column and Givens rotations on the device, stops the scenes that
  // have converged, and advances j.
  void enqueue_batch_step(double* V, double* Z, int* jp, int maxit) {
    const Mask mk{bb.act, S.scene_of_vertex.as<int32_t>()};
    const SegTiles T = tiles();
    switch (precond) {
      case NCPADJ_PRECOND_NONE:
        launch_seg_copy_step(T, V, true, w, false, N, jp, m, bb.act, nullptr, st);
        break;
      case NCPADJ_PRECOND_JACOBI:
        launch_seg_copy_step(T, V, true, w, false, N, jp, m, bb.act, dinv, st);
        break;
      default: {
        launch_sinv_half1_idx(sinv, V, N, jp, mixed ? nullptr : t3, mixed ? w32 : nullptr, st, mk);
        if (precond == NCPADJ_PRECOND_WOODBURY && cnc) {
          const int32_t* ip = S.iperm.as<int32_t>();
          launch_path_gather(cnc, cvx, ip, sinv, t3, mixed ? w32 : nullptr, cfr, ccd, transpose, sc, st, mk);
          cap_apply_all(sc, tc, bb.act);
          launch_path_scatter(cnc, cvx, ip, sinv, cfr, tc, -h * h, t3, mixed ? w32 : nullptr, st, mk);
        }
        if (mixed) launch_sinv_half2_32(sinv, w32, w, st, mk);
        else launch_sinv_half2(sinv, t3, w, st, mk);
      }
    }
    // Z_j = P^{-1} V_j (and its double-float pairs for the mixed product); V_{j+1} = A Z_j
    launch_seg_copy_step(T, w, false, Z, true, N, jp, m, bb.act, nullptr, st, mixed ? zsplit : nullptr);
    if (mixed)
      launch_bsr_spmv_ff(nv, S.row_ptr.as<int32_t>(), S.col.as<int32_t>(), S.bsr32.as<float>(), zsplit, V, N, jp, st,
                         mk);
    else
      launch_bsr_spmv_idx(nv, S.row_ptr.as<int32_t>(), S.col.as<int32_t>(), S.bsr64.as<double>(), nullptr, w, V, N,
                          jp, st, mk);
    const int g2 = m + 1, gn = 2 * (m + 1);
    launch_seg_dot_step(T, V, N, jp, m, false, bb.act, bb.partial, bb.cnt, bb.K, bb.gsb, bb.gstride, 0, st);
    launch_seg_axpy_step(T, V, N, jp, m, bb.act, bb.gsb, bb.gstride, 0, st);
    launch_seg_dot_step(T, V, N, jp, m, false, bb.act, bb.partial, bb.cnt, bb.K, bb.gsb, bb.gstride, g2, st);
    launch_seg_axpy_step(T, V, N, jp, m, bb.act, bb.gsb, bb.gstride, g2, st);
    launch_seg_dot_step(T, V, N, jp, m, true, bb.act, bb.partial, bb.cnt, bb.K, bb.gsb, bb.gstride, gn, st);
    launch_seg_normalize_step(T, V, N, jp, m, bb.act, bb.gsb, bb.gstride, gn, st);
    launch_seg_givens(bb.ns, jp, m, bb.act, bb.gsb, bb.gstride, bb.H, bb.cs, bb.sn, bb.g, bb.kk, bb.iters, bb.tol,
                      maxit, S.bmap_dev, st);
  }
  cudaGraphExec_t batch_step_graph(double* V, double* Z, int* jp, int maxit) {
    std::vector<uintptr_t> key = step_key();
    for (uintptr_t v : {(uintptr_t)precond, (uintptr_t)maxit, (uintptr_t)S.bwork.p, (uintptr_t)S.segt.p,
                        (uintptr_t)S.bmap_dev, (uintptr_t)S.iperm.p})
      key.push_back(v);
    for (int v : blk_scene) key.push_back((uintptr_t)v);
    if (S.bstep_exec && key == S.bstep_key) return S.bstep_exec;
    if (S.bstep_exec) {
      cudaGraphExecDestroy(S.bstep_exec);
      S.bstep_exec = nullptr;
    }
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    const int64_t l0 = g_launches;
    enqueue_batch_step(V, Z, jp, maxit);
    S.bstep_launches = (int)(g_launches - l0);
    g_launches = l0;
    const cudaError_t ce = cudaStreamEndCapture(st, &gr);
    if (ce != cudaSuccess || !gr) {
      cudaGetLastError();
      if (gr) cudaGraphDestroy(gr);
      return nullptr;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    S.bstep_exec = ex;
    S.bstep_key = key;
    return ex;
  }

  // Solve B x = b scene by scene: every mesh of the batch runs its own right-preconditioned
  // flexible GMRES(m) (Sec. 4.4) to ||b_s - B_s x_s|| <= rtol ||b_s||, x0 = 0, with its own inner
  // products, Hessenberg matrix, restarts and stopping test; a mesh that has converged drops out
  // of every later launch.  The host only launches steps (one captured graph per step off the
  // legacy default stream) and reads, per step, how many meshes are still active.
  // Returns the largest per-scene iteration count; per-scene counts and final true relative
  // residuals go to S.last_iters / S.last_rel.
  int solve_batched(double rtol, int max_iters) {
    const int ns = bb.ns;
    const SegTiles T = tiles();
    double* V = S.gmres.as<double>();
    double* Z = S.fgmres.as<double>();
    int* jp = S.gstep.as<int>();
    int* nact_dev = S.bmap_dev;
    int* notdone_dev = S.bmap_dev + kMaxRestart;
    volatile int* nact_h = S.bmap_host;
    volatile int* notdone_h = S.bmap_host + kMaxRestart;
    const Mask mcyc{bb.cyc, S.scene_of_vertex.as<int32_t>()};
    NCPADJ_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * N, st));
    NCPADJ_CUDA_TRY(cudaMemsetAsync(bb.cnt, 0, sizeof(unsigned) * (size_t)ns * bb.K, st));
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    launch_seg_init(ns, bb.cyc, bb.done, bb.iters, st);
    launch_seg_sq(T, r, bb.cyc, bb.partial, bb.cnt, bb.K, m + 2, bb.rr, st);
    launch_seg_restart(ns, m, true, bb.cyc, bb.act, bb.done, bb.kk, bb.iters, max_iters, bb.rr, bb.bnorm, bb.tol,
                       rtol, bb.relres, bb.g, jp, flags, notdone_dev, st);
    launch_seg_start(T, r, bb.act, bb.g, m, V, st);
    NCPADJ_CUDA_TRY(cudaEventRecord(S.bev[0], st));
    NCPADJ_CUDA_TRY(cudaEventSynchronize(S.bev[0]));
    int notdone = *notdone_h;
    cudaGraphExec_t gx = batch_step_graph(V, Z, jp, max_iters);
    constexpr int kAhead = 3;  // steps in flight (< the 4 events of S.bev)
    for (int cycle = 0; notdone > 0 && cycle <= max_iters; ++cycle) {
      int launched = 0, seen = 0;
      while (seen < m) {
        while (launched < m && launched < seen + kAhead) {
          if (gx) {
            NCPADJ_CUDA_TRY(cudaGraphLaunch(gx, st));
            g_launches += S.bstep_launches;
          } else {
            enqueue_batch_step(V, Z, jp, max_iters);
          }
          NCPADJ_CUDA_TRY(cudaEventRecord(S.bev[launched & 3], st));
          ++launched;
        }
        NCPADJ_CUDA_TRY(cudaEventSynchronize(S.bev[seen & 3]));
        const int na = nact_h[seen];
        ++seen;
        if (na == 0) break;
      }
      // end of the cycle: x_s += Z_s y_s, true residual, restart or stop, scene by scene
      launch_seg_backsolve(ns, m, bb.cyc, bb.kk, bb.H, bb.g, bb.y, st);
      launch_seg_combine(T, Z, N, m, bb.cyc, bb.kk, bb.y, x, st);
      matvec(x, w, mcyc);
      launch_seg_resid(T, b, w, bb.cyc, r, st);
      launch_seg_sq(T, r, bb.cyc, bb.partial, bb.cnt, bb.K, m + 2, bb.rr, st);
      launch_seg_restart(ns, m, false, bb.cyc, bb.act, bb.done, bb.kk, bb.iters, max_iters, bb.rr, bb.bnorm, bb.tol,
                         rtol, bb.relres, bb.g, jp, flags, notdone_dev, st);
      launch_seg_start(T, r, bb.act, bb.g, m, V, st);
      NCPADJ_CUDA_TRY(cudaEventRecord(S.bev[0], st));
      NCPADJ_CUDA_TRY(cudaEventSynchronize(S.bev[0]));
      notdone = *notdone_h;
    }
    NCPADJ_CUDA_TRY(cudaGetLastError());
    S.last_iters.assign(ns, 0);
    S.last_rel.assign(ns, 0.0);
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.last_iters.data(), bb.iters, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.last_rel.data(), bb.relres, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    (void)nact_dev;
    int most = 0;
    for (int v : S.last_iters) most = std::max(most, v);
    return most;
  }

  double dot_host(const double* a, const double* bb) {
    launch_multi_dot(N, 1, a, N, bb, partial, scal, st);
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.scal_host, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    return S.scal_host[0];
  }

  // Solve B x = b (B the assembled matrix) to ||b - B x|| <= rtol ||b||, x0 = 0.
  // CG for symmetric systems, else right-preconditioned restarted GMRES with classical
  // Gram-Schmidt applied twice.  Returns the number of iterations; *rel = final true residual.
  int solve(int solver, double rtol, int max_iters, double* rel, double* bnorm_out) {
    NCPADJ_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * N, st));
    const double bnorm = std::sqrt(dot_host(b, b));
    *bnorm_out = bnorm;
    int iters = 0;
    if (bnorm > 0.0 && std::isfinite(bnorm)) {
      const double tol = rtol * bnorm;
      if (solver == NCPADJ_SOLVER_CG) {
        double* p = w;
        double* rr = S.gmres.as<double>();
        double* zz = rr + N;
        double* Ap = rr + 2 * (size_t)N;
        double* s2 = scal + 8;  // rz_old, rz_new, pAp, alpha
        auto cg_start = [&]() {  // z = P^{-1} rr, p = z, rz = rr . z
          apply_precond(rr, zz);
          NCPADJ_CUDA_TRY(cudaMemcpyAsync(p, zz, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
          launch_multi_dot(N, 1, rr, N, zz, partial, s2 + 0, st);
        };
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(rr, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        cg_start();
        for (iters = 1; iters <= max_iters; ++iters) {
          matvec(p, Ap);
          launch_multi_dot(N, 1, p, N, Ap, partial, s2 + 2, st);
          launch_cg_alpha(s2 + 0, s2 + 2, s2 + 3, st);
          launch_cg_update_xr(N, s2 + 3, p, Ap, x, rr, st);
          const double rn = std::sqrt(dot_host(rr, rr));
          if (!std::isfinite(rn)) break;
          if (rn <= tol) {
            // the recursively updated residual drifts away from b - B x on ill-conditioned systems
            // (stiff bindings); stop only when the true residual is there too, else restart from it
            matvec(x, r);
            launch_axpby(N, 1.0, b, -1.0, r, r, st);
            const double rt = std::sqrt(dot_host(r, r));
            if (!std::isfinite(rt) || rt <= tol || iters >= max_iters) break;
            NCPADJ_CUDA_TRY(cudaMemcpyAsync(rr, r, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
            cg_start();
            continue;
          }
          apply_precond(rr, zz);
          launch_multi_dot(N, 1, rr, N, zz, partial, s2 + 1, st);
          launch_cg_update_p(N, s2 + 1, s2 + 0, zz, p, st);
          launch_copy_scalar(s2 + 1, s2 + 0, st);
        }
        iters = std::min(iters, max_iters);
      } else if (solver == NCPADJ_SOLVER_SEMI_IMPLICIT) {
        // The stationary splitting of the forward solver's local-global structure (Sec. 4.4, Eq.
        // semi-implicit): P x^{k+1} = (P - B) x^k + b, i.e. preconditioned Richardson
        // x^{k+1} = x^k + P^{-1} (b - B x^k).  With the elastic preconditioner (P = A) this is the
        // baseline the paper compares against; it converges only when the spectral radius of
        // I - P^{-1} B is below 1 and is stopped when the residual grows past 1e6 ||b||.
        double* zz = S.gmres.as<double>();
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        for (iters = 1; iters <= max_iters; ++iters) {
          apply_precond(r, zz);
          launch_axpby(N, 1.0, x, 1.0, zz, x, st);
          matvec(x, w);
          launch_axpby(N, 1.0, b, -1.0, w, r, st);
          const double rn = std::sqrt(dot_host(r, r));
          if (!std::isfinite(rn) || rn <= tol || rn > 1e6 * bnorm) break;
        }
        iters = std::min(iters, max_iters);
      } else if (solver == NCPADJ_SOLVER_BICGSTAB) {
        // right-preconditioned BiCGSTAB (van der Vorst 1992): iterates on A P^{-1} u = b and
        // accumulates x = P^{-1} u directly.  Scalars on the host (one synchronisation per inner
        // product); the seven vectors in columns of the GMRES buffer, t and s adjacent so that one
        // call gives t.t and s.t.  A breakdown ends the loop; the true residual below decides.
        double* G = S.gmres.as<double>();
        double *rh = G, *p = G + N, *v = G + 2 * (size_t)N, *ph = G + 3 * (size_t)N, *t = G + 4 * (size_t)N,
               *s = G + 5 * (size_t)N, *sh = G + 6 * (size_t)N;
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(rh, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
        for (iters = 1; iters <= max_iters; ++iters) {
          const double rho = dot_host(rh, r);
          if (!std::isfinite(rho) || rho == 0.0) break;
          if (iters == 1) {
            NCPADJ_CUDA_TRY(cudaMemcpyAsync(p, r, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
          } else {
            const double beta = (rho / rho_old) * (alpha / omega);
            launch_axpby(N, 1.0, p, -omega, v, p, st);  // p - omega v
            launch_axpby(N, 1.0, r, beta, p, p, st);    // r + beta (p - omega v)
          }
          apply_precond(p, ph);
          matvec(ph, v);
          const double rv = dot_host(rh, v);
          if (!std::isfinite(rv) || rv == 0.0) break;
          alpha = rho / rv;
          launch_axpby(N, 1.0, r, -alpha, v, s, st);  // s = r - alpha v
          const double sn = std::sqrt(dot_host(s, s));
          if (!std::isfinite(sn)) break;
          if (sn <= tol) {
            launch_axpby(N, 1.0, x, alpha, ph, x, st);
            break;
          }
          apply_precond(s, sh);
          matvec(sh, t);
          launch_multi_dot(N, 2, t, N, t, partial, scal + 12, st);  // t.t, s.t
          NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.scal_host + 12, scal + 12, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
          NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
          const double tt = S.scal_host[12], ts = S.scal_host[13];
          omega = (tt > 0.0 && std::isfinite(tt)) ? ts / tt : 0.0;
          launch_axpby(N, 1.0, x, alpha, ph, x, st);
          launch_axpby(N, 1.0, x, omega, sh, x, st);
          launch_axpby(N, 1.0, s, -omega, t, r, st);  // r = s - omega t
          rho_old = rho;
          const double rn = std::sqrt(dot_host(r, r));
          if (!std::isfinite(rn) || rn <= tol || omega == 0.0) break;
        }
        iters = std::min(iters, max_iters);
      } else {
        // Arnoldi vectors on the device; the small Hessenberg least-squares problem (Givens
        // rotations, triangular solve) on the host, which reads the Gram-Schmidt coefficients of
        // each iteration in one copy together with the convergence check.
        double* V = S.gmres.as<double>();  // (m+1) x N
        const bool flexible = flexible_gmres();
        double* Z = flexible ? S.fgmres.as<double>() : nullptr;
        double* gs = V + (size_t)(m + 1) * N;  // [0..m]: first-pass, [m+1..2m+1]: second-pass, [2m+2]: norm
        double* ydev = gs + 2 * (m + 1) + 1;
        double* nrm2 = scal + 5;
        std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m), hbuf(2 * (m + 1) + 1);
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        double beta = bnorm;
        for (;;) {
          launch_axpby(N, 1.0 / beta, r, 0.0, nullptr, V, st);
          std::fill(g.begin(), g.end(), 0.0);
          g[0] = beta;
          int k = 0;
          // Arnoldi step j on the device; its coefficients go to pinned slot j % 2 with an event.
          // The host enqueues step j + 1 before it reads step j's coefficients, so the GPU never
          // waits for the host's Givens update (a converged cycle leaves one step unused).
          const size_t slot = 2 * (size_t)(m + 1) + 1;
          cudaGraphExec_t gx = step_graph(V, gs, nrm2);
          if (gx) NCPADJ_CUDA_TRY(cudaMemsetAsync(S.gstep.p, 0, sizeof(int), st));
          auto enqueue_step = [&](int j) {
            if (gx) {
              NCPADJ_CUDA_TRY(cudaGraphLaunch(gx, st));
              g_launches += S.step_launches;
              NCPADJ_CUDA_TRY(cudaEventRecord(S.gs_ev[j & 1], st));
              return;
            }
            double* vn = V + (size_t)(j + 1) * N;
            double* zj = flexible ? Z + (size_t)j * N : w;
            apply_precond(V + (size_t)j * N, zj);
            matvec(zj, vn);
            launch_multi_dot(N, j + 1, V, N, vn, partial, gs, st);
            launch_multi_axpy(N, j + 1, V, N, gs, vn, st);
            launch_multi_dot(N, j + 1, V, N, vn, partial, gs + (m + 1), st);
            launch_multi_axpy(N, j + 1, V, N, gs + (m + 1), vn, st);
            launch_multi_dot(N, 1, vn, N, vn, partial, nrm2, st);
            launch_normalize(N, vn, nrm2, vn, gs + 2 * (m + 1), st);
            NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.gs_host + (j & 1) * slot, gs, sizeof(double) * slot,
                                            cudaMemcpyDeviceToHost, st));
            NCPADJ_CUDA_TRY(cudaEventRecord(S.gs_ev[j & 1], st));
          };
          enqueue_step(0);
          for (int j = 0; j < m; ++j) {
            if (j + 1 < m && iters + 1 < max_iters) enqueue_step(j + 1);
            NCPADJ_CUDA_TRY(cudaEventSynchronize(S.gs_ev[j & 1]));
            const double* gh = (gx ? S.gs_map_host : S.gs_host) + (j & 1) * slot;
            double* h = &H[(size_t)(m + 1) * j];
            for (int i = 0; i <= j; ++i) h[i] = gh[i] + gh[m + 1 + i];
            h[j + 1] = gh[2 * (m + 1)];
            for (int i = 0; i < j; ++i) {  // previous rotations
              const double t = cs[i] * h[i] + sn[i] * h[i + 1];
              h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
              h[i] = t;
            }
            const double rr = std::hypot(h[j], h[j + 1]);
            cs[j] = rr > 0 ? h[j] / rr : 1.0;
            sn[j] = rr > 0 ? h[j + 1] / rr : 0.0;
            h[j] = rr;
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++iters;
            k = j + 1;
            const double res_est = std::fabs(g[j + 1]);
            if (!std::isfinite(res_est) || res_est <= tol || iters >= max_iters) break;
          }
          for (int i = k - 1; i >= 0; --i) {  // H(0:k,0:k) y = g(0:k)
            double t = g[i];
            for (int jj = i + 1; jj < k; ++jj) t -= H[(size_t)(m + 1) * jj + i] * y[jj];
            y[i] = t / H[(size_t)(m + 1) * i + i];
          }
          NCPADJ_CUDA_TRY(cudaMemcpyAsync(ydev, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
          if (flexible) {
            launch_combine(N, k, Z, N, ydev, w, st);
          } else {
            launch_combine(N, k, V, N, ydev, r, st);
            apply_precond(r, w);
          }
          launch_axpby(N, 1.0, x, 1.0, w, x, st);
          matvec(x, w);
          launch_axpby(N, 1.0, b, -1.0, w, r, st);
          beta = std::sqrt(dot_host(r, r));
          if (!std::isfinite(beta) || beta <= tol || iters >= max_iters) break;
        }
      }
    }
    NCPADJ_CUDA_TRY(cudaGetLastError());
    matvec(x, w);
    launch_axpby(N, 1.0, b, -1.0, w, r, st);
    const double rfinal = std::sqrt(dot_host(r, r));
    *rel = (bnorm > 0) ? rfinal / bnorm : 0.0;
    return iters;
  }
};

void read_flags(Scene& S, cudaStream_t st) {
  NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.flags_host, S.flags.as<int>(), FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, st));
  NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
}

void check_contacts(Scene& S, int nc, const int32_t* cvertex, const int32_t* region, int nreg, cudaStream_t st) {
  if (!nc) return;
  launch_check_contacts(nc, cvertex, region, S.nv, nreg, S.flags.as<int>(), st);
  read_flags(S, st);
  NCPADJ_REQUIRE(S.flags_host[FLAG_BADINDEX] == 0, "a contact vertex or region id is out of range");
}

// the call's bilateral bindings into the engine's inputs, after checking their vertex ids and
// compliances on the device (the flags were cleared at the start of the call)
void take_bindings(Scene& S, const ncpadj_bindings* bd, bool host_mem, Inputs& in, cudaStream_t st) {
  if (!bd) return;
  NCPADJ_REQUIRE(bd->n_bindings >= 0, "n_bindings < 0");
  if (bd->n_bindings == 0) return;
  const bool bary = bd->tet || bd->bary;
  NCPADJ_REQUIRE(!bary || (bd->tet && bd->bary), "bindings need both tet and bary, or neither");
  NCPADJ_REQUIRE(!bary || S.nvpe == 4, "bindings inside elements (tet, bary) need a tet scene");
  NCPADJ_REQUIRE((bary || bd->vertex) && bd->target && bd->compliance,
                 "binding arrays vertex (or tet and bary), target, compliance are required");
  NCPADJ_REQUIRE(!host_mem, "bindings need options.memory = NCPADJ_MEM_DEVICE");
  if (bary)
    launch_check_bindings_bary(bd->n_bindings, bd->tet, bd->bary, bd->compliance, S.nt, S.flags.as<int>(), st);
  else
    launch_check_bindings(bd->n_bindings, bd->vertex, bd->compliance, S.nv, S.flags.as<int>(), st);
  read_flags(S, st);
  NCPADJ_REQUIRE(S.flags_host[FLAG_BADINDEX] == 0,
                 bary ? "a binding tet is out of range, a weight is not finite or a compliance is not positive"
                      : "a binding vertex is out of range or a compliance is not positive");
  in.nbind = bd->n_bindings;
  in.bvertex = bary ? nullptr : bd->vertex;
  in.btarget = bd->target;
  in.bcompliance = bd->compliance;
  in.btet = bary ? bd->tet : nullptr;
  in.bbary = bary ? bd->bary : nullptr;
}

int pick_solver(int requested, int nc, const double* mu, bool host_mem, cudaStream_t st) {
  if (requested != NCPADJ_SOLVER_AUTO) return requested;
  bool frictionless = true;
  if (nc) {
    std::vector<double> muh(nc);
    if (host_mem) std::memcpy(muh.data(), mu, nc * sizeof(double));
    else {
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(muh.data(), mu, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
      NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    }
    for (double v : muh) frictionless = frictionless && (v == 0.0);
  }
  return frictionless ? NCPADJ_SOLVER_CG : NCPADJ_SOLVER_GMRES;
}

void validate_options(const ncpadj_options& opt) {
  NCPADJ_REQUIRE(opt.eps > 0 && opt.rtol > 0 && opt.max_iters > 0 && opt.gmres_restart > 0 && opt.gmres_restart <= 512,
                 "bad options (eps, rtol, max_iters, gmres_restart)");
  NCPADJ_REQUIRE(opt.cap_drop >= 0 && std::isfinite(opt.cap_drop), "bad option cap_drop (must be finite, >= 0)");
  NCPADJ_REQUIRE(opt.precond >= 0 && opt.precond <= 3 && opt.solver >= 0 && opt.solver <= 4, "bad precond/solver");
  NCPADJ_REQUIRE(opt.memory == NCPADJ_MEM_DEVICE || opt.memory == NCPADJ_MEM_HOST, "bad memory kind");
  NCPADJ_REQUIRE(opt.precision == NCPADJ_FP64 || opt.precision == NCPADJ_MIXED, "bad precision");
  NCPADJ_REQUIRE(opt.cap_precision == NCPADJ_FP64 || opt.cap_precision == NCPADJ_MIXED ||
                     opt.cap_precision == NCPADJ_TF32X3 || opt.cap_precision == NCPADJ_REFINED,
                 "bad cap_precision");
  NCPADJ_REQUIRE(opt.cap_block >= 0, "bad cap_block");
}

void raise_flags(const int* fh) {
  if (fh[FLAG_INVERTED]) throw Error{NCPADJ_ERR_INVERTED_ELEMENT, "a tet has det F <= 0 at the given state"};
  if (fh[FLAG_TIMEOUT]) throw Error{NCPADJ_ERR_TIMEOUT, "a grid barrier of the capacitance inversion timed out"};
  if (fh[FLAG_DOMAIN]) throw Error{NCPADJ_ERR_CONTACT_DOMAIN, "a frictional contact has zero slip and zero tangential force"};
  if (fh[FLAG_SINGULAR]) throw Error{NCPADJ_ERR_NONFINITE, "the contact capacitance is singular"};
  if (fh[FLAG_NONFINITE]) throw Error{NCPADJ_ERR_NONFINITE, "non-finite values in the solve"};
}

}  // namespace

// ------------------------------------------------------------------------------------------
// the adjoint step
// ------------------------------------------------------------------------------------------
static ncpadj_status adjoint_step(ncpadj_ctx_s* ctx, ncpadj_scene_s* sc, const ncpadj_contacts* ct,
                                  const ncpadj_state* state, const ncpadj_seed* seed, const ncpadj_options* opt_in,
                                  ncpadj_grads* grads, ncpadj_stats* stats, cudaStream_t st) {
  NCPADJ_REQUIRE(ctx && sc, "NULL context or scene");
  NCPADJ_REQUIRE(state && seed && state->q && state->q_prev && seed->dL_dq, "state.q, state.q_prev and seed.dL_dq are required");
  NCPADJ_REQUIRE(!grads || !grads->dL_dact || sc->s.fibre.p,
                 "dL_dact requested but the scene has no fibres (ncpadj_scene_set_fibres)");
  NCPADJ_REQUIRE(!grads || (!grads->dL_dbinding_target && !grads->dL_dcompliance) ||
                     (state->bindings && state->bindings->n_bindings > 0),
                 "binding gradients requested but state.bindings holds no bindings");
  ncpadj_options opt;
  if (opt_in) opt = *opt_in;
  else ncpadj_options_default(&opt);
  validate_options(opt);
  Scene& S = sc->s;
  const int nc = ct ? ct->n_contacts : 0;
  NCPADJ_REQUIRE(nc >= 0, "n_contacts < 0");
  if (nc > 0) {
    NCPADJ_REQUIRE(ct->vertex && ct->frame && ct->d_n && ct->mu, "contact arrays vertex, frame, d_n, mu are required");
    NCPADJ_REQUIRE(state->lambda, "state.lambda is required when there are contacts");
    NCPADJ_REQUIRE(ct->n_regions >= 1, "n_regions must be >= 1");
  }
  const int nv = S.nv, nt = S.nt, N = 3 * nv;
  const int nreg = (nc > 0) ? ct->n_regions : 1;
  const bool host_mem = opt.memory == NCPADJ_MEM_HOST;
  if (nc && host_mem)
    for (int c = 0; c < nc; ++c) NCPADJ_REQUIRE(ct->vertex[c] >= 0 && ct->vertex[c] < nv, "contact vertex out of range");

  const long long launches0 = g_launches;
  Engine E(S, ctx->c, st);
  Inputs& in = E.in;
  // ---- stage inputs ----
  if (host_mem) {
    size_t nd = (size_t)4 * N + (size_t)nc * (3 + 9 + 1 + 2 + 1);
    S.io.ensure(nd * sizeof(double) + (size_t)2 * nc * sizeof(int32_t) + 64);
    double* p = S.io.as<double>();
    auto put = [&](const double* src, size_t n) -> const double* {
      if (!src || n == 0) return nullptr;
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(p, src, n * sizeof(double), cudaMemcpyHostToDevice, st));
      const double* r = p;
      p += n;
      return r;
    };
    in.q = put(state->q, N);
    in.q_prev = put(state->q_prev, N);
    in.dL_dq = put(seed->dL_dq, N);
    in.dL_dv = put(seed->dL_dv, N);
    if (nc) {
      in.lambda = put(state->lambda, 3 * (size_t)nc);
      in.frame = put(ct->frame, 9 * (size_t)nc);
      in.d_n = put(ct->d_n, nc);
      in.d_f = put(ct->d_f, 2 * (size_t)nc);
      in.mu = put(ct->mu, nc);
      int32_t* ip = reinterpret_cast<int32_t*>(S.io.as<double>() + nd);
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(ip, ct->vertex, nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      in.cvertex = ip;
      if (ct->region) {
        NCPADJ_CUDA_TRY(cudaMemcpyAsync(ip + nc, ct->region, nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        in.region = ip + nc;
      }
    }
  } else {
    in.q = state->q;
    in.q_prev = state->q_prev;
    in.dL_dq = seed->dL_dq;
    in.dL_dv = seed->dL_dv;
    if (nc) {
      in.lambda = state->lambda;
      in.frame = ct->frame;
      in.d_n = ct->d_n;
      in.d_f = ct->d_f;
      in.mu = ct->mu;
      in.cvertex = ct->vertex;
      in.region = ct->region;
    }
  }
  int solver = pick_solver(opt.solver, nc, nc ? ct->mu : nullptr, host_mem, st);
  E.mixed = opt.precision == NCPADJ_MIXED;
  E.cap_fp32 = opt.cap_precision != NCPADJ_FP64;
  E.cap_tc = opt.cap_precision == NCPADJ_TF32X3 || opt.cap_precision == NCPADJ_REFINED;
  E.cap_refine = opt.cap_precision == NCPADJ_REFINED;
  E.cap_block = opt.cap_block;
  E.cap_drop = opt.cap_drop;
  int* flags = E.flags;
  NCPADJ_CUDA_TRY(cudaMemsetAsync(flags, 0, FLAG_COUNT * sizeof(int), st));
  check_contacts(S, nc, in.cvertex, in.region, nreg, st);  // before anything indexes with the ids
  take_bindings(S, state->bindings, host_mem, in, st);
  // a batch scene solves every mesh by its own GMRES (CG and BiCGSTAB, when asked for by name,
  // run over the union with the scaled right-hand side below)
  E.batch_mode = S.n_scenes > 1 && (opt.solver == NCPADJ_SOLVER_AUTO || opt.solver == NCPADJ_SOLVER_GMRES);
  E.workspace(nc, opt.gmres_restart, opt.precond);
  // an inner iterative capacitance solve makes the preconditioner vary: flexible GMRES only
  if (!E.sup_c0.empty() && opt.precond == NCPADJ_PRECOND_WOODBURY) solver = NCPADJ_SOLVER_GMRES;
  if (E.batch_mode) solver = NCPADJ_SOLVER_GMRES;
  E.transpose = 1;
  NCPADJ_CUDA_TRY(cudaEventRecord(S.ev[0], st));
  E.assemble(in.q, in.q_prev, in.lambda, opt.eps);
  NCPADJ_CUDA_TRY(cudaEventRecord(S.ev[1], st));
  E.setup_precond();
  NCPADJ_CUDA_TRY(cudaEventRecord(S.ev[2], st));
  launch_rhs(N, in.dL_dq, in.dL_dv, 1.0 / S.h, E.b, st);
  double rel = 0, bnorm = 0;
  // a batch holds independent systems: scale each scene's right-hand side to unit norm so that the
  // union's relative residual bounds every scene's (the scaling is undone on z afterwards)
  std::vector<double> scale;
  double rtol = opt.rtol;
  const bool union_scaled = S.n_scenes > 1 && !E.batch_mode;
  if (union_scaled) {
    const int ns = S.n_scenes;
    S.sceneval.ensure(sizeof(double) * 2 * (size_t)ns);
    double* sq = S.sceneval.as<double>();
    NCPADJ_CUDA_TRY(cudaMemsetAsync(sq, 0, sizeof(double) * ns, st));
    launch_scene_sq(nv, E.b, S.scene_of_vertex.as<int32_t>(), sq, st);
    std::vector<double> h_sq(ns);
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(h_sq.data(), sq, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    scale.assign(2 * (size_t)ns, 1.0);
    int nz = 0;
    for (int i = 0; i < ns; ++i)
      if (h_sq[i] > 0) {
        scale[i] = 1.0 / std::sqrt(h_sq[i]);
        scale[ns + i] = std::sqrt(h_sq[i]);
        ++nz;
      }
    rtol = opt.rtol / std::sqrt((double)std::max(nz, 1));
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(sq, scale.data(), sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, st));
    launch_scale_by_scene(nv, E.b, S.scene_of_vertex.as<int32_t>(), sq, st);
  }
  int iters = 0;
  if (E.batch_mode) {
    iters = E.solve_batched(rtol, opt.max_iters);
    for (double v : S.last_rel) rel = std::max(rel, std::isfinite(v) ? v : INFINITY);
    bnorm = 1.0;
  } else {
    S.last_iters.clear();
    S.last_rel.clear();
    iters = E.solve(solver, rtol, opt.max_iters, &rel, &bnorm);
  }
  if (union_scaled)
    launch_scale_by_scene(nv, E.x, S.scene_of_vertex.as<int32_t>(), S.sceneval.as<double>() + S.n_scenes, st);
  NCPADJ_CUDA_TRY(cudaEventRecord(S.ev[3], st));

  // ---- contractions ----
  ncpadj_grads go{};
  if (grads) go = *grads;
  if (host_mem) {  // device staging for outputs
    size_t need = (size_t)4 * N + 2 * (size_t)nt + nreg + nc + S.n_scenes + 16;
    S.c_in.ensure(need * sizeof(double));
    double* p = S.c_in.as<double>();
    auto slot = [&](double* user, size_t n) -> double* {
      if (!user) return nullptr;
      double* r = p;
      p += n;
      return r;
    };
    go.dL_dbend = slot(grads ? grads->dL_dbend : nullptr, S.n_scenes);
    go.dL_dq_prev = slot(grads ? grads->dL_dq_prev : nullptr, N);
    go.dL_dv_prev = slot(grads ? grads->dL_dv_prev : nullptr, N);
    go.dL_dfext = slot(grads ? grads->dL_dfext : nullptr, N);
    go.z = slot(grads ? grads->z : nullptr, N);
    go.dL_dE = slot(grads ? grads->dL_dE : nullptr, nt);
    go.dL_dnu = slot(grads ? grads->dL_dnu : nullptr, nt);
    go.dL_dmu = slot(grads ? grads->dL_dmu : nullptr, nreg);
    go.dL_dmu_contact = slot(grads ? grads->dL_dmu_contact : nullptr, nc);
  }
  if (go.dL_dmu) NCPADJ_CUDA_TRY(cudaMemsetAsync(go.dL_dmu, 0, sizeof(double) * nreg, st));
  ContractArgs ka{nv, S.nvpe == 4 ? nt : 0, nc, S.h, E.x, S.massd.as<double>(), in.dL_dv, S.tets.as<int32_t>(),
                  S.gvec.as<double>(), S.tetdata.as<double>(), S.lame_d.as<double>(), in.cvertex, in.frame,
                  S.cdata.as<double>(), in.region, go.dL_dq_prev, go.dL_dv_prev, go.dL_dfext, go.dL_dE, go.dL_dnu,
                  go.dL_dmu, go.dL_dmu_contact};
  launch_contractions(ka, st);
  if (S.nvpe == 3) {
    ka.nt = nt;
    launch_contract_tri(ka, st);
  }
  if (go.dL_dbend) {
    if (S.n_bend)
      launch_bend_grad(S.n_scenes, S.bend_eoff.as<int32_t>(), S.bend_idx.as<int32_t>(), S.bend_coef.as<double>(), in.q,
                       E.x, S.h, go.dL_dbend, st);
    else
      NCPADJ_CUDA_TRY(cudaMemsetAsync(go.dL_dbend, 0, sizeof(double) * S.n_scenes, st));
  }
  float* dact = nullptr;
  if (grads && grads->dL_dact) {
    if (host_mem) {
      S.actf.ensure(std::max(sizeof(float) * (size_t)nt, sizeof(double) * N));
      dact = S.actf.as<float>();
    } else {
      dact = grads->dL_dact;
    }
    launch_act_grad(nt, S.tets.as<int32_t>(), S.gvec.as<double>(), S.vol.as<double>(), S.fibre.as<double>(), E.x, S.h,
                    dact, st);
  }
  if (in.nbind && grads && (grads->dL_dbinding_target || grads->dL_dcompliance)) {
    if (in.btet)
      launch_binding_grad_bary(in.nbind, in.btet, S.tets.as<int32_t>(), in.bbary, in.btarget, in.bcompliance, in.q,
                               E.x, S.h, grads->dL_dbinding_target, grads->dL_dcompliance, st);
    else
      launch_binding_grad(in.nbind, in.bvertex, in.btarget, in.bcompliance, in.q, E.x, S.h, grads->dL_dbinding_target,
                          grads->dL_dcompliance, st);
  }
  if (go.z) NCPADJ_CUDA_TRY(cudaMemcpyAsync(go.z, E.x, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  launch_nonfinite_check(N, E.x, flags, st);
  NCPADJ_CUDA_TRY(cudaGetLastError());
  NCPADJ_CUDA_TRY(cudaEventRecord(S.ev[4], st));
  if (host_mem && grads) {
    auto back = [&](double* user, double* dev, size_t n) {
      if (user && dev) NCPADJ_CUDA_TRY(cudaMemcpyAsync(user, dev, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    };
    back(grads->dL_dq_prev, go.dL_dq_prev, N);
    back(grads->dL_dv_prev, go.dL_dv_prev, N);
    back(grads->dL_dfext, go.dL_dfext, N);
    back(grads->z, go.z, N);
    back(grads->dL_dE, go.dL_dE, nt);
    back(grads->dL_dnu, go.dL_dnu, nt);
    back(grads->dL_dmu, go.dL_dmu, nreg);
    back(grads->dL_dmu_contact, go.dL_dmu_contact, nc);
    back(grads->dL_dbend, go.dL_dbend, S.n_scenes);
    if (dact) NCPADJ_CUDA_TRY(cudaMemcpyAsync(grads->dL_dact, dact, sizeof(float) * nt, cudaMemcpyDeviceToHost, st));
  }
  read_flags(S, st);
  if (stats) {
    stats->iterations = iters;
    stats->solver_used = solver;
    stats->n_contacts = nc;
    stats->capacitance_dim = (opt.precond == NCPADJ_PRECOND_WOODBURY) ? 3 * E.cnc : 0;
    stats->capacitance_blocks = (opt.precond == NCPADJ_PRECOND_WOODBURY && nc) ? (int32_t)E.blk_c0.size() : 0;
    stats->inner_iterations = E.inner_iters;
    stats->rel_residual = rel;
    float ms[5] = {0, 0, 0, 0, 0};
    cudaEventElapsedTime(&ms[0], S.ev[0], S.ev[4]);
    cudaEventElapsedTime(&ms[1], S.ev[0], S.ev[1]);
    cudaEventElapsedTime(&ms[2], S.ev[1], S.ev[2]);
    cudaEventElapsedTime(&ms[3], S.ev[2], S.ev[3]);
    cudaEventElapsedTime(&ms[4], S.ev[3], S.ev[4]);
    stats->ms_total = ms[0];
    stats->ms_assemble = ms[1];
    stats->ms_setup = ms[2];
    stats->ms_krylov = ms[3];
    stats->ms_contract = ms[4];
    float mc = 0;
    if (E.cap_timed) cudaEventElapsedTime(&mc, S.ev[6], S.ev[7]);
    stats->ms_cap_inverse = mc;
    stats->kernel_launches = g_launches - launches0;
  }
  raise_flags(S.flags_host);
  if (!std::isfinite(rel)) throw Error{NCPADJ_ERR_NONFINITE, "non-finite residual"};
  if (!(rel <= rtol * 1.0000001) && bnorm > 0) {
    char msg[160];
    snprintf(msg, sizeof msg, "Krylov stopped at relative residual %.3e (rtol %.1e) after %d iterations", rel, rtol,
             iters);
    throw Error{NCPADJ_ERR_NOT_CONVERGED, msg};
  }
  return NCPADJ_OK;
}

// ------------------------------------------------------------------------------------------
// the batched adjoint: per-scene arrays in, per-scene arrays out, one union solve in between
// ------------------------------------------------------------------------------------------
// Copy tables of one call (pinned host memory, uploaded in one copy): FP64 copies, int32 id copies
// with offsets, FP32 copies, and the [ns + 1] contact / vertex / region offsets.
struct CopyTable {
  std::vector<const void*> fsrc, isrc, ssrc;
  std::vector<void*> fdst, idst, sdst;
  std::vector<int64_t> fcnt, icnt, scnt;
  std::vector<int32_t> iadd;
  void f64(const double* src, double* dst, int64_t n) {
    if (!src || !dst || n <= 0) return;
    fsrc.push_back(src);
    fdst.push_back(dst);
    fcnt.push_back(n);
  }
  void ids(const int32_t* src, int32_t* dst, int64_t n, int32_t add) {
    if (!dst || n <= 0) return;
    isrc.push_back(src);
    idst.push_back(dst);
    icnt.push_back(n);
    iadd.push_back(add);
  }
  void f32(const float* src, float* dst, int64_t n) {
    if (!src || !dst || n <= 0) return;
    ssrc.push_back(src);
    sdst.push_back(dst);
    scnt.push_back(n);
  }
  // uploads the tables (and the offsets) and launches the copies
  void run(Scene& S, const std::vector<int32_t>& offsets, const int32_t** off_dev, cudaStream_t st) {
    const size_t nf = fsrc.size(), ni = isrc.size(), ns = ssrc.size(), no = offsets.size();
    const size_t bytes = 8 * (3 * nf + 3 * ni + 3 * ns) + 4 * (ni + no) + 64;
    if (S.btab_host_bytes < bytes) {
      if (S.btab_host) cudaFreeHost(S.btab_host);
      S.btab_host = nullptr;
      S.btab_host_bytes = 0;
      NCPADJ_CUDA_TRY(cudaMallocHost(&S.btab_host, bytes));
      S.btab_host_bytes = bytes;
    }
    S.btab.ensure(bytes);
    char* h = static_cast<char*>(S.btab_host);
    char* d = S.btab.as<char>();
    size_t o = 0;
    auto put = [&](const void* src, size_t nbytes) {
      if (nbytes) std::memcpy(h + o, src, nbytes);
      const size_t at = o;
      o += (nbytes + 7) & ~size_t(7);
      return d + at;
    };
    char* fs = put(fsrc.data(), 8 * nf);
    char* fd = put(fdst.data(), 8 * nf);
    char* fc = put(fcnt.data(), 8 * nf);
    char* is = put(isrc.data(), 8 * ni);
    char* id = put(idst.data(), 8 * ni);
    char* ic = put(icnt.data(), 8 * ni);
    char* ia = put(iadd.data(), 4 * ni);
    char* ss = put(ssrc.data(), 8 * ns);
    char* sd = put(sdst.data(), 8 * ns);
    char* sc = put(scnt.data(), 8 * ns);
    char* of = put(offsets.data(), 4 * no);
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(d, h, o, cudaMemcpyHostToDevice, st));
    launch_gather_f64((int)nf, reinterpret_cast<const double* const*>(fs), reinterpret_cast<double* const*>(fd),
                      reinterpret_cast<const int64_t*>(fc), st);
    launch_gather_ids((int)ni, reinterpret_cast<const int32_t* const*>(is), reinterpret_cast<int32_t* const*>(id),
                      reinterpret_cast<const int64_t*>(ic), reinterpret_cast<const int32_t*>(ia), st);
    launch_gather_f32((int)ns, reinterpret_cast<const float* const*>(ss), reinterpret_cast<float* const*>(sd),
                      reinterpret_cast<const int64_t*>(sc), st);
    if (off_dev) *off_dev = reinterpret_cast<const int32_t*>(of);
    NCPADJ_CUDA_TRY(cudaGetLastError());
  }
};

static ncpadj_status adjoint_batch(ncpadj_ctx_s* ctx, ncpadj_scene_s* sc, int ns, const ncpadj_contacts* cts,
                                   const ncpadj_state* states, const ncpadj_seed* seeds, const ncpadj_options* opt_in,
                                   ncpadj_grads* grads, ncpadj_stats* stats, cudaStream_t st) {
  NCPADJ_REQUIRE(ctx && sc, "NULL context or scene");
  Scene& S = sc->s;
  NCPADJ_REQUIRE(ns == S.n_scenes, "n_scenes must equal the number of meshes of the batch scene");
  NCPADJ_REQUIRE(states && seeds, "states and seeds are required");
  ncpadj_options opt;
  if (opt_in) opt = *opt_in;
  else ncpadj_options_default(&opt);
  validate_options(opt);
  if (opt.solver != NCPADJ_SOLVER_AUTO && opt.solver != NCPADJ_SOLVER_GMRES)
    throw Error{NCPADJ_ERR_UNSUPPORTED, "the batched adjoint runs GMRES per scene (solver AUTO or GMRES)"};
  const bool host_mem = opt.memory == NCPADJ_MEM_HOST;
  // sizes, offsets and what is present
  std::vector<int32_t> coff(ns + 1, 0), roff(ns + 1, 0);
  bool any_df = false, any_dv = false, any_region = false;
  for (int s = 0; s < ns; ++s) {
    const ncpadj_state& x = states[s];
    NCPADJ_REQUIRE(x.q && x.q_prev && seeds[s].dL_dq, "every scene needs state.q, state.q_prev and seed.dL_dq");
    NCPADJ_REQUIRE(!x.bindings || x.bindings->n_bindings == 0, "bindings are not supported in a batched call");
    const int n = cts ? cts[s].n_contacts : 0;
    NCPADJ_REQUIRE(n >= 0, "n_contacts < 0");
    if (n > 0) {
      NCPADJ_REQUIRE(cts[s].vertex && cts[s].frame && cts[s].d_n && cts[s].mu,
                     "contact arrays vertex, frame, d_n, mu are required");
      NCPADJ_REQUIRE(x.lambda, "state.lambda is required when a scene has contacts");
      NCPADJ_REQUIRE(cts[s].n_regions >= 1, "n_regions must be >= 1");
      any_df = any_df || cts[s].d_f;
      any_region = any_region || cts[s].region;
    }
    any_dv = any_dv || seeds[s].dL_dv;
    coff[s + 1] = coff[s] + n;
    roff[s + 1] = roff[s] + (n > 0 ? cts[s].n_regions : 0);
    if (grads && grads[s].dL_dact) NCPADJ_REQUIRE(S.fibre.p, "dL_dact requested but the scene has no fibres");
  }
  const int nc = coff[ns], nreg = std::max(roff[ns], 1), N = 3 * S.nv, nt = S.nt;
  auto want = [&](size_t off) {  // does some scene ask for the output at byte offset off of ncpadj_grads
    if (!grads) return false;
    for (int s = 0; s < ns; ++s)
      if (*reinterpret_cast<void* const*>(reinterpret_cast<const char*>(&grads[s]) + off)) return true;
    return false;
  };
  const bool w_dq = want(offsetof(ncpadj_grads, dL_dq_prev)), w_dv = want(offsetof(ncpadj_grads, dL_dv_prev)),
             w_df = want(offsetof(ncpadj_grads, dL_dfext)), w_z = want(offsetof(ncpadj_grads, z)),
             w_E = want(offsetof(ncpadj_grads, dL_dE)), w_nu = want(offsetof(ncpadj_grads, dL_dnu)),
             w_mu = want(offsetof(ncpadj_grads, dL_dmu)), w_muc = want(offsetof(ncpadj_grads, dL_dmu_contact)),
             w_act = want(offsetof(ncpadj_grads, dL_dact)), w_bend = want(offsetof(ncpadj_grads, dL_dbend));
  // union staging: inputs, then outputs
  const size_t nd = 8 * (size_t)N + 17 * (size_t)nc + 2 * (size_t)nt + nreg + ns + 64;
  S.bio.ensure(sizeof(double) * nd + sizeof(float) * (size_t)nt + 256);
  double* p = S.bio.as<double>();
  auto take = [&](size_t n) {
    double* r = p;
    p += n;
    return r;
  };
  double *uq = take(N), *uqp = take(N), *udq = take(N), *udv = take(N), *ulam = take(3 * (size_t)nc),
         *ufr = take(9 * (size_t)nc), *udn = take(nc), *udf = take(2 * (size_t)nc), *umu = take(nc);
  double *o_dq = take(N), *o_dv = take(N), *o_df = take(N), *o_z = take(N), *o_E = take(nt), *o_nu = take(nt),
         *o_mu = take(nreg), *o_muc = take(nc), *o_bend = take(ns);
  float* o_act = reinterpret_cast<float*>(p + 8);
  S.bio_ids.ensure(sizeof(int32_t) * (4 * (size_t)nc + 64));
  int32_t* uvert = S.bio_ids.as<int32_t>();
  int32_t* ureg = uvert + nc;
  int32_t* raw = ureg + nc;  // host-memory calls: the ids as given, before their offsets
  if (any_dv) NCPADJ_CUDA_TRY(cudaMemsetAsync(udv, 0, sizeof(double) * N, st));
  if (any_df && nc) NCPADJ_CUDA_TRY(cudaMemsetAsync(udf, 0, sizeof(double) * 2 * nc, st));
  CopyTable in;
  auto h2d = [&](const void* src, void* dst, size_t bytes) {
    if (src && bytes) NCPADJ_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
  };
  for (int s = 0; s < ns; ++s) {
    const size_t v0 = 3 * (size_t)S.voff[s], nv3 = 3 * (size_t)(S.voff[s + 1] - S.voff[s]);
    const int n = coff[s + 1] - coff[s];
    const size_t c0 = coff[s];
    const ncpadj_state& x = states[s];
    if (host_mem) {
      h2d(x.q, uq + v0, 8 * nv3);
      h2d(x.q_prev, uqp + v0, 8 * nv3);
      h2d(seeds[s].dL_dq, udq + v0, 8 * nv3);
      h2d(seeds[s].dL_dv, udv + v0, 8 * nv3);
      if (n) {
        h2d(x.lambda, ulam + 3 * c0, 24 * (size_t)n);
        h2d(cts[s].frame, ufr + 9 * c0, 72 * (size_t)n);
        h2d(cts[s].d_n, udn + c0, 8 * (size_t)n);
        h2d(cts[s].d_f, udf + 2 * c0, 16 * (size_t)n);
        h2d(cts[s].mu, umu + c0, 8 * (size_t)n);
        h2d(cts[s].vertex, raw + c0, 4 * (size_t)n);
        h2d(cts[s].region, raw + nc + c0, 4 * (size_t)n);
        in.ids(raw + c0, uvert + c0, n, S.voff[s]);
        if (any_region) in.ids(cts[s].region ? raw + nc + c0 : nullptr, ureg + c0, n, roff[s]);
      }
    } else {
      in.f64(x.q, uq + v0, nv3);
      in.f64(x.q_prev, uqp + v0, nv3);
      in.f64(seeds[s].dL_dq, udq + v0, nv3);
      in.f64(seeds[s].dL_dv, udv + v0, nv3);
      if (n) {
        in.f64(x.lambda, ulam + 3 * c0, 3 * (int64_t)n);
        in.f64(cts[s].frame, ufr + 9 * c0, 9 * (int64_t)n);
        in.f64(cts[s].d_n, udn + c0, n);
        in.f64(cts[s].d_f, udf + 2 * c0, 2 * (int64_t)n);
        in.f64(cts[s].mu, umu + c0, n);
        in.ids(cts[s].vertex, uvert + c0, n, S.voff[s]);
        if (any_region) in.ids(cts[s].region, ureg + c0, n, roff[s]);
      }
    }
  }
  std::vector<int32_t> offs;
  offs.insert(offs.end(), coff.begin(), coff.end());
  offs.insert(offs.end(), S.voff.begin(), S.voff.end());
  offs.insert(offs.end(), roff.begin(), roff.end());
  const int32_t* off_dev = nullptr;
  in.run(S, offs, &off_dev, st);
  if (nc) {  // every contact must name a vertex (and region) of its own scene
    int* flags = S.flags.as<int>();
    NCPADJ_CUDA_TRY(cudaMemsetAsync(flags, 0, FLAG_COUNT * sizeof(int), st));
    launch_check_batch_ids(nc, uvert, any_region ? ureg : nullptr, ns, off_dev, off_dev + (ns + 1),
                           off_dev + 2 * (ns + 1), flags, st);
    read_flags(S, st);
    NCPADJ_REQUIRE(S.flags_host[FLAG_BADINDEX] == 0,
                   "a contact vertex or region id is out of its scene's range");
  }
  // one adjoint over the union
  ncpadj_contacts uc{nc, uvert, ufr, udn, any_df ? udf : nullptr, umu, any_region ? ureg : nullptr, nreg};
  ncpadj_state us{uq, uqp, nc ? ulam : nullptr, nullptr};
  ncpadj_seed ud{udq, any_dv ? udv : nullptr};
  ncpadj_grads ug{};
  ug.dL_dq_prev = w_dq ? o_dq : nullptr;
  ug.dL_dv_prev = w_dv ? o_dv : nullptr;
  ug.dL_dfext = w_df ? o_df : nullptr;
  ug.z = w_z ? o_z : nullptr;
  ug.dL_dE = w_E ? o_E : nullptr;
  ug.dL_dnu = w_nu ? o_nu : nullptr;
  ug.dL_dmu = (w_mu && nc) ? o_mu : nullptr;
  ug.dL_dmu_contact = (w_muc && nc) ? o_muc : nullptr;
  ug.dL_dact = w_act ? o_act : nullptr;
  ug.dL_dbend = w_bend ? o_bend : nullptr;
  ncpadj_options uo = opt;
  uo.memory = NCPADJ_MEM_DEVICE;
  uo.solver = NCPADJ_SOLVER_GMRES;
  ncpadj_stats ust{};
  ncpadj_status status = NCPADJ_OK;
  std::string status_msg;
  try {
    adjoint_step(ctx, sc, nc ? &uc : nullptr, &us, &ud, &uo, &ug, &ust, st);
  } catch (const Error& e) {
    // NOT_CONVERGED still delivers the outputs (the last iterate); anything else ends the call
    if (e.status != NCPADJ_ERR_NOT_CONVERGED) throw;
    status = e.status;
    status_msg = e.msg;
  }
  // outputs back to each scene's own arrays
  if (grads) {
    CopyTable out;
    auto d2h = [&](void* dst, const void* src, size_t bytes) {
      if (dst && src && bytes) NCPADJ_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
    };
    for (int s = 0; s < ns; ++s) {
      const ncpadj_grads& gs = grads[s];
      const size_t v0 = 3 * (size_t)S.voff[s], nv3 = 3 * (size_t)(S.voff[s + 1] - S.voff[s]);
      const size_t t0 = S.toff[s], nts = S.toff[s + 1] - S.toff[s];
      const size_t c0 = coff[s], n = coff[s + 1] - coff[s], r0 = roff[s], nr = roff[s + 1] - roff[s];
      if (host_mem) {
        d2h(gs.dL_dq_prev, o_dq + v0, 8 * nv3);
        d2h(gs.dL_dv_prev, o_dv + v0, 8 * nv3);
        d2h(gs.dL_dfext, o_df + v0, 8 * nv3);
        d2h(gs.z, o_z + v0, 8 * nv3);
        d2h(gs.dL_dE, o_E + t0, 8 * nts);
        d2h(gs.dL_dnu, o_nu + t0, 8 * nts);
        if (n) d2h(gs.dL_dmu, o_mu + r0, 8 * nr);
        if (n) d2h(gs.dL_dmu_contact, o_muc + c0, 8 * n);
        d2h(gs.dL_dact, o_act + t0, 4 * nts);
        d2h(gs.dL_dbend, o_bend + s, 8);
      } else {
        out.f64(o_dq + v0, gs.dL_dq_prev, nv3);
        out.f64(o_dv + v0, gs.dL_dv_prev, nv3);
        out.f64(o_df + v0, gs.dL_dfext, nv3);
        out.f64(o_z + v0, gs.z, nv3);
        out.f64(o_E + t0, gs.dL_dE, nts);
        out.f64(o_nu + t0, gs.dL_dnu, nts);
        if (n) out.f64(o_mu + r0, gs.dL_dmu, nr);
        if (n) out.f64(o_muc + c0, gs.dL_dmu_contact, n);
        out.f32(o_act + t0, gs.dL_dact, nts);
        out.f64(o_bend + s, gs.dL_dbend, 1);
      }
    }
    if (!host_mem) out.run(S, {}, nullptr, st);
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (stats)
    for (int s = 0; s < ns; ++s) {
      stats[s] = ust;
      stats[s].iterations = s < (int)S.last_iters.size() ? S.last_iters[s] : ust.iterations;
      stats[s].rel_residual = s < (int)S.last_rel.size() ? S.last_rel[s] : ust.rel_residual;
      stats[s].n_contacts = coff[s + 1] - coff[s];
    }
  if (status != NCPADJ_OK) throw Error{status, status_msg};
  return NCPADJ_OK;
}

// ------------------------------------------------------------------------------------------
// the forward step (produces the converged state the adjoint differentiates)
// ------------------------------------------------------------------------------------------
static ncpadj_status forward_step(ncpadj_ctx_s* ctx, ncpadj_scene_s* sc, const ncpadj_contacts* ct,
                                  const ncpadj_forward_input* fin, const ncpadj_options* opt_in, double newton_tol,
                                  int max_newton, double* q_out, double* lambda_out, ncpadj_forward_stats* stats,
                                  cudaStream_t st) {
  NCPADJ_REQUIRE(ctx && sc && fin && fin->q_prev && q_out, "NULL required argument");
  NCPADJ_REQUIRE(!fin->act || sc->s.fibre.p, "actuation given but the scene has no fibres (ncpadj_scene_set_fibres)");
  NCPADJ_REQUIRE(newton_tol > 0 && max_newton > 0, "newton_tol and max_newton must be positive");
  ncpadj_options opt;
  if (opt_in) opt = *opt_in;
  else ncpadj_options_default(&opt);
  validate_options(opt);
  if (opt.memory != NCPADJ_MEM_DEVICE) throw Error{NCPADJ_ERR_UNSUPPORTED, "the forward step takes device memory"};
  Scene& S = sc->s;
  const int nc = ct ? ct->n_contacts : 0;
  if (nc) {
    NCPADJ_REQUIRE(ct->vertex && ct->frame && ct->d_n && ct->mu && ct->n_regions >= 1, "incomplete contact arrays");
    NCPADJ_REQUIRE(lambda_out, "lambda_out is required when there are contacts");
  }
  const int nv = S.nv, N = 3 * nv;
  Engine E(S, ctx->c, st);
  E.in.cvertex = nc ? ct->vertex : nullptr;
  E.in.frame = nc ? ct->frame : nullptr;
  E.in.d_n = nc ? ct->d_n : nullptr;
  E.in.d_f = nc ? ct->d_f : nullptr;
  E.in.mu = nc ? ct->mu : nullptr;
  E.in.region = nc ? ct->region : nullptr;
  E.in.q_prev = fin->q_prev;
  int solver = pick_solver(opt.solver, nc, E.in.mu, false, st);
  // the Newton solves run in FP64; the capacitance (a preconditioner only) follows cap_precision
  E.cap_fp32 = opt.cap_precision != NCPADJ_FP64;
  E.cap_tc = opt.cap_precision == NCPADJ_TF32X3 || opt.cap_precision == NCPADJ_REFINED;
  E.cap_refine = opt.cap_precision == NCPADJ_REFINED;
  E.cap_block = opt.cap_block;
  E.cap_drop = opt.cap_drop;
  int* flags = E.flags;
  NCPADJ_CUDA_TRY(cudaMemsetAsync(flags, 0, FLAG_COUNT * sizeof(int), st));
  check_contacts(S, nc, E.in.cvertex, E.in.region, nc ? ct->n_regions : 1, st);  // before any indexing
  take_bindings(S, fin->bindings, false, E.in, st);
  E.workspace(nc, opt.gmres_restart, opt.precond);
  if (!E.sup_c0.empty() && opt.precond == NCPADJ_PRECOND_WOODBURY) solver = NCPADJ_SOLVER_GMRES;
  E.transpose = 0;
  S.fwd.ensure(sizeof(double) * (4 * (size_t)N + 3 * (size_t)std::max(nc, 1) + 4 * (size_t)std::max(nc, 1)) +
               sizeof(int) * std::max(nc, 1) + 64);
  double* qt = S.fwd.as<double>();  // inertial prediction
  double* q = qt + N;               // current iterate (q_out holds trials)
  double* R = q + N;
  double* Rt = R + N;
  double* lam = Rt + N;                         // [3 nc]
  double* slip_old = lam + 3 * std::max(nc, 1);  // [2 nc]
  double* slip_new = slip_old + 2 * std::max(nc, 1);
  int* loaded = reinterpret_cast<int*>(slip_new + 2 * std::max(nc, 1));
  cudaEvent_t e0 = S.ev[0], e1 = S.ev[5];
  NCPADJ_CUDA_TRY(cudaEventRecord(e0, st));
  const double* f_total = fin->f_ext;
  if (fin->act) {  // f_ext + f_act
    S.actf.ensure(sizeof(double) * N);
    double* fa = S.actf.as<double>();
    if (fin->f_ext) NCPADJ_CUDA_TRY(cudaMemcpyAsync(fa, fin->f_ext, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    else NCPADJ_CUDA_TRY(cudaMemsetAsync(fa, 0, sizeof(double) * N, st));
    launch_act_force(S.nt, S.tets.as<int32_t>(), S.gvec.as<double>(), S.vol.as<double>(), fin->act,
                     S.fibre.as<double>(), fa, st);
    f_total = fa;
  }
  launch_predict(nv, fin->q_prev, fin->v_prev, f_total, S.massd.as<double>(), fin->gravity[0], fin->gravity[1],
                 fin->gravity[2], S.h, qt, st);
  NCPADJ_CUDA_TRY(cudaMemcpyAsync(q, qt, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  double fscale = 0, start_gap = 0;
  {
    const double g2 = fin->gravity[0] * fin->gravity[0] + fin->gravity[1] * fin->gravity[1] + fin->gravity[2] * fin->gravity[2];
    double mmax = 0, m2 = 0;
    for (double mv : S.mass) {
      mmax = std::max(mmax, mv);
      m2 += mv * mv;
    }
    fscale = S.h * S.h * std::sqrt(m2 * std::max(g2, 1e-30));
    start_gap = 10.0 * opt.eps * opt.eps / std::max(mmax * std::sqrt(std::max(g2, 1e-30)), 1e-300);
    launch_lift(nc, E.in.cvertex, E.in.frame, E.in.d_n, start_gap, q, fin->q_prev, E.in.d_f, st);
  }
  // residual at a point: R = M (q - qt) + h^2 sum w G^T (G q - p) - h^2 J^T lambda(q); returns ||R||^2 or
  // +inf if the point leaves the local-solve domain (or turns a loaded slip, when asked)
  auto evaluate = [&](const double* qq, double* RR, double* slip, bool check_turn) -> double {
    NCPADJ_CUDA_TRY(cudaMemsetAsync(flags + FLAG_INFEASIBLE, 0, 2 * sizeof(int), st));
    launch_inertia(nv, S.massd.as<double>(), qq, qt, RR, st);
    if (S.nvpe == 3) {
      launch_tri_force(S.nt, S.tets.as<int32_t>(), S.gvec.as<double>(), S.vol.as<double>(), S.mu.as<double>(),
                       S.lam.as<double>(), S.model_ptr(), qq, S.h, RR, flags, st);
      launch_bend_force(S.n_bend, S.bend_idx.as<int32_t>(), S.bend_coef.as<double>(), S.bend_kb.as<double>(), qq,
                        S.h, RR, st);
    } else {
      launch_tet_force(S.nt, S.tets.as<int32_t>(), S.gvec.as<double>(), S.vol.as<double>(), S.mu.as<double>(),
                       S.lam.as<double>(), S.model_ptr(), qq, S.h, RR, flags, st);
    }
    if (E.in.nbind && E.in.btet)
      launch_binding_force_bary(E.in.nbind, E.in.btet, S.tets.as<int32_t>(), E.in.bbary, E.in.btarget,
                                E.in.bcompliance, qq, S.h, RR, st);
    else if (E.in.nbind)
      launch_binding_force(E.in.nbind, E.in.bvertex, E.in.btarget, E.in.bcompliance, qq, S.h, RR, st);
    if (nc) {
      ContactArgs ca = E.contact_args(qq, fin->q_prev, nullptr, opt.eps);
      // the loaded mask belongs to the accepted iterate: trial points (check_turn) leave it alone
      launch_local_contact(ca, lam, slip, check_turn ? nullptr : loaded, RR, st);
      if (check_turn) launch_turn_check(nc, slip_old, slip, loaded, flags, E.in.cvertex, RR, st);
    }
    launch_multi_dot(N, 1, RR, N, RR, E.partial, E.scal + 6, st);
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.scal_host + 6, E.scal + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
    read_flags(S, st);
    if (S.flags_host[FLAG_INVERTED] || S.flags_host[FLAG_INFEASIBLE] || S.flags_host[FLAG_TURN]) {
      S.flags_host[FLAG_INVERTED] = 0;
      NCPADJ_CUDA_TRY(cudaMemsetAsync(flags + FLAG_INVERTED, 0, sizeof(int), st));
      return INFINITY;
    }
    return S.scal_host[6];
  };
  // A batch holds independent scenes: each gets its own line search (a failing or slowly converging
  // scene must not hold the others back).  The residual kernels poison the rows of a vertex whose
  // tet inverted, whose contact left the local-solve domain or whose slip turned, so the
  // per-scene squared norms tell which scenes failed.
  const int ns = S.n_scenes;
  const bool batch = ns > 1;
  std::vector<double> phis(ns, 0.0), phits(ns, 0.0), tsc(ns, 1.0);
  const int32_t* sov = S.scene_of_vertex.as<int32_t>();
  if (batch) S.sceneval.ensure(sizeof(double) * 2 * (size_t)ns);
  auto evaluate_scenes = [&](const double* qq, double* RR, double* slip, bool check_turn,
                             std::vector<double>& out) -> double {
    evaluate(qq, RR, slip, check_turn);  // flags are global: the poisoned rows carry the per-scene news
    NCPADJ_CUDA_TRY(cudaMemsetAsync(flags + FLAG_INVERTED, 0, sizeof(int), st));
    double* sq = S.sceneval.as<double>();
    NCPADJ_CUDA_TRY(cudaMemsetAsync(sq, 0, sizeof(double) * ns, st));
    launch_scene_sq(nv, RR, sov, sq, st);
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(out.data(), sq, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    double tot = 0.0;
    for (double& v : out) {
      if (!std::isfinite(v)) v = INFINITY;
      tot += v;
    }
    return tot;
  };
  auto set_scene_t = [&](const std::vector<double>& t) {
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(S.sceneval.as<double>() + ns, t.data(), sizeof(double) * ns,
                                    cudaMemcpyHostToDevice, st));
  };
  double phi = batch ? evaluate_scenes(q, R, slip_old, false, phis) : evaluate(q, R, slip_old, false);
  {
    // large forces on light vertices can put the inertial prediction outside the domain (an
    // inverted tet): back off towards q_prev, q = q_prev + t (qt - q_prev), t = 1/2, 1/4, ...
    // (per scene in a batch)
    if (!batch) {
      double t = 1.0;
      for (int k = 0; !std::isfinite(phi) && k < 40; ++k) {
        t *= 0.5;
        launch_axpby(N, 1.0 - t, fin->q_prev, t, qt, q, st);
        launch_lift(nc, E.in.cvertex, E.in.frame, E.in.d_n, start_gap, q, fin->q_prev, E.in.d_f, st);
        phi = evaluate(q, R, slip_old, false);
      }
    } else {
      launch_axpby(N, 1.0, qt, -1.0, fin->q_prev, Rt, st);  // Rt = qt - q_prev (scratch)
      std::vector<double> t(ns, 1.0);
      for (int k = 0; !std::isfinite(phi) && k < 40; ++k) {
        for (int i = 0; i < ns; ++i)
          if (!std::isfinite(phis[i])) t[i] *= 0.5;
        set_scene_t(t);
        launch_step_by_scene(nv, fin->q_prev, Rt, sov, S.sceneval.as<double>() + ns, q, st);
        launch_lift(nc, E.in.cvertex, E.in.frame, E.in.d_n, start_gap, q, fin->q_prev, E.in.d_f, st);
        phi = evaluate_scenes(q, R, slip_old, false, phis);
      }
    }
  }
  if (!std::isfinite(phi)) throw Error{NCPADJ_ERR_CONTACT_DOMAIN, "no feasible start point for the Newton solve"};
  int it = 0, kry = 0;
  for (it = 0; it < max_newton; ++it) {
    if (std::sqrt(phi) <= newton_tol * fscale) break;
    // Newton matrix script_A at q with the local multipliers (loaded mask recomputed here)
    if (nc) {
      ContactArgs ca = E.contact_args(q, fin->q_prev, nullptr, opt.eps);
      launch_local_contact(ca, lam, slip_old, loaded, Rt, st);  // refresh lam/slips/loaded at q (Rt scratch)
    }
    E.assemble(q, fin->q_prev, lam, opt.eps);
    E.setup_precond();
    launch_axpby(N, -1.0, R, 0.0, nullptr, E.b, st);
    double rel = 0, bn = 0;
    kry += E.solve(solver, std::min(1e-10, 1e-3), opt.max_iters, &rel, &bn);
    read_flags(S, st);
    raise_flags(S.flags_host);
    // backtracking line search on ||R|| (per scene in a batch)
    double t = 1.0, phit = INFINITY;
    bool ok = false;
    if (!batch) {
      for (int ls = 0; ls < 40; ++ls) {
        launch_axpby(N, 1.0, q, t, E.x, q_out, st);
        phit = evaluate(q_out, Rt, slip_new, true);
        if (phit <= (1.0 - 1e-4 * t) * phi) {
          ok = true;
          break;
        }
        t *= 0.5;
      }
    } else {
      std::vector<char> acc(ns, 0);
      std::fill(tsc.begin(), tsc.end(), 1.0);
      bool settled = false;
      for (int ls = 0; ls < 40 && !settled; ++ls) {
        set_scene_t(tsc);
        launch_step_by_scene(nv, q, E.x, sov, S.sceneval.as<double>() + ns, q_out, st);
        phit = evaluate_scenes(q_out, Rt, slip_new, true, phits);
        settled = true;
        for (int i = 0; i < ns; ++i) {
          if (acc[i]) continue;
          if (phits[i] <= (1.0 - 1e-4 * tsc[i]) * phis[i]) {
            acc[i] = 1;
            ok = true;
          } else {
            tsc[i] *= 0.5;
            settled = false;
          }
        }
      }
      if (ok && !settled) {  // scenes that found no decrease stay where they are
        for (int i = 0; i < ns; ++i)
          if (!acc[i]) tsc[i] = 0.0;
        set_scene_t(tsc);
        launch_step_by_scene(nv, q, E.x, sov, S.sceneval.as<double>() + ns, q_out, st);
        phit = evaluate_scenes(q_out, Rt, slip_new, true, phits);
      }
      if (ok) phis = phits;
    }
    if (!ok) break;  // no decrease possible: rounding floor
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(q, q_out, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(R, Rt, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(slip_old, slip_new, sizeof(double) * 2 * nc, cudaMemcpyDeviceToDevice, st));
    phi = phit;
  }
  // outputs at the final iterate
  NCPADJ_CUDA_TRY(cudaMemcpyAsync(q_out, q, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  phi = evaluate(q, R, slip_new, false);
  if (nc) NCPADJ_CUDA_TRY(cudaMemcpyAsync(lambda_out, lam, sizeof(double) * 3 * nc, cudaMemcpyDeviceToDevice, st));
  NCPADJ_CUDA_TRY(cudaEventRecord(e1, st));
  NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
  const double res = std::sqrt(phi) / fscale;
  if (stats) {
    stats->newton_iters = it;
    stats->krylov_iters = kry;
    stats->residual = res;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    stats->ms_total = ms;
  }
  if (!std::isfinite(res)) throw Error{NCPADJ_ERR_NONFINITE, "non-finite forward residual"};
  if (res > 1e3 * newton_tol) {
    char msg[96];
    snprintf(msg, sizeof msg, "forward Newton stopped at relative residual %.3e", res);
    throw Error{NCPADJ_ERR_NOT_CONVERGED, msg};
  }
  return NCPADJ_OK;
}

}  // namespace ncpadj

// ------------------------------------------------------------------------------------------
// C-ABI
// ------------------------------------------------------------------------------------------
using namespace ncpadj;

extern "C" {

const char* ncpadj_version(void) { return "ncpadj 0.1 (sm_103a)"; }

const char* ncpadj_status_string(ncpadj_status s) {
  switch (s) {
    case NCPADJ_OK: return "OK";
    case NCPADJ_ERR_INVALID_ARG: return "INVALID_ARG";
    case NCPADJ_ERR_CUDA: return "CUDA";
    case NCPADJ_ERR_OOM: return "OOM";
    case NCPADJ_ERR_INVERTED_ELEMENT: return "INVERTED_ELEMENT";
    case NCPADJ_ERR_NOT_CONVERGED: return "NOT_CONVERGED";
    case NCPADJ_ERR_NONFINITE: return "NONFINITE";
    case NCPADJ_ERR_TIMEOUT: return "TIMEOUT";
    case NCPADJ_ERR_NOT_FACTORED: return "NOT_FACTORED";
    case NCPADJ_ERR_UNSUPPORTED: return "UNSUPPORTED";
    case NCPADJ_ERR_CONTACT_DOMAIN: return "CONTACT_DOMAIN";
  }
  return "UNKNOWN";
}

const char* ncpadj_last_error(void) { return g_last_error.c_str(); }

void ncpadj_options_default(ncpadj_options* o) {
  if (!o) return;
  o->eps = 1e-4;
  o->rtol = 1e-8;
  o->max_iters = 2000;
  o->gmres_restart = 64;
  o->cap_drop = 1e-2;
  o->precision = NCPADJ_FP64;
  o->precond = NCPADJ_PRECOND_WOODBURY;
  o->solver = NCPADJ_SOLVER_AUTO;
  o->memory = NCPADJ_MEM_DEVICE;
  o->cap_precision = NCPADJ_FP64;
  o->cap_block = 0;
}

ncpadj_status ncpadj_ctx_create(int device, ncpadj_ctx* out) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(out, "out is NULL");
    *out = nullptr;
    int n = 0;
    NCPADJ_CUDA_TRY(cudaGetDeviceCount(&n));
    NCPADJ_REQUIRE(device >= 0 && device < n, "no CUDA device " + std::to_string(device));
    NCPADJ_CUDA_TRY(cudaSetDevice(device));
    auto* c = new ncpadj_ctx_s();
    c->c.device = device;
    cudaDeviceGetAttribute(&c->c.sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&c->c.coop_ok, cudaDevAttrCooperativeLaunch, device);
    try {
      noalloc_prepare(device);  // the allocation-free solve's static scratch is loaded now, not in that call
    } catch (...) {
      delete c;
      throw;
    }
    *out = c;
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_INVALID_ARG, e.what()});
  }
}

void ncpadj_ctx_destroy(ncpadj_ctx ctx) { delete ctx; }

ncpadj_status ncpadj_scene_create(ncpadj_ctx ctx, const ncpadj_scene_desc* desc, ncpadj_scene* out) {
  g_last_error.clear();
  ncpadj_scene_s* s = nullptr;
  try {
    NCPADJ_REQUIRE(ctx && desc && out, "NULL argument");
    *out = nullptr;
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    s = new ncpadj_scene_s();
    s->ctx = ctx;
    const MeshSpec m = spec_of(*desc);
    build_scene(s->s, &m, 1);
    keep_geometry(s->s, &m, 1);
    *out = s;
    return NCPADJ_OK;
  } catch (const Error& e) {
    ncpadj_scene_destroy(s);
    return fail(e);
  } catch (const std::exception& e) {
    ncpadj_scene_destroy(s);
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_scene_create_batch(ncpadj_ctx ctx, int32_t n_scenes, const ncpadj_scene_desc* descs,
                                        ncpadj_scene* out) {
  g_last_error.clear();
  ncpadj_scene_s* s = nullptr;
  try {
    NCPADJ_REQUIRE(ctx && descs && out && n_scenes >= 1, "NULL argument or n_scenes < 1");
    *out = nullptr;
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    s = new ncpadj_scene_s();
    s->ctx = ctx;
    std::vector<MeshSpec> m(n_scenes);
    for (int i = 0; i < n_scenes; ++i) m[i] = spec_of(descs[i]);
    build_scene(s->s, m.data(), n_scenes);
    keep_geometry(s->s, m.data(), n_scenes);
    *out = s;
    return NCPADJ_OK;
  } catch (const Error& e) {
    ncpadj_scene_destroy(s);
    return fail(e);
  } catch (const std::exception& e) {
    ncpadj_scene_destroy(s);
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_scene_create_shells(ncpadj_ctx ctx, int32_t n_scenes, const ncpadj_shell_desc* descs,
                                         ncpadj_scene* out) {
  g_last_error.clear();
  ncpadj_scene_s* s = nullptr;
  try {
    NCPADJ_REQUIRE(ctx && descs && out && n_scenes >= 1, "NULL argument or n_scenes < 1");
    *out = nullptr;
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    s = new ncpadj_scene_s();
    s->ctx = ctx;
    std::vector<MeshSpec> m(n_scenes);
    for (int i = 0; i < n_scenes; ++i) m[i] = spec_of(descs[i]);
    build_scene(s->s, m.data(), n_scenes);
    keep_geometry(s->s, m.data(), n_scenes);
    *out = s;
    return NCPADJ_OK;
  } catch (const Error& e) {
    ncpadj_scene_destroy(s);
    return fail(e);
  } catch (const std::exception& e) {
    ncpadj_scene_destroy(s);
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_scene_set_bending(ncpadj_scene scene, const double* bend, void* stream) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(scene && bend, "NULL argument");
    NCPADJ_REQUIRE(scene->ctx, "scene without a context");
    Scene& S = scene->s;
    NCPADJ_REQUIRE(S.nvpe == 3, "bending stiffness belongs to shell scenes (ncpadj_scene_create_shells)");
    for (int i = 0; i < S.n_scenes; ++i)
      NCPADJ_REQUIRE(bend[i] >= 0 && std::isfinite(bend[i]), "mesh " + std::to_string(i) + ": need bend >= 0");
    NCPADJ_CUDA_TRY(cudaSetDevice(scene->ctx->c.device));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    refactor_scene(S, S.mat_E.data(), S.mat_nu.data(), bend);
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_scene_get_bending(ncpadj_scene scene, double* bend) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(scene && bend, "NULL argument");
    const Scene& S = scene->s;
    for (int i = 0; i < S.n_scenes; ++i) bend[i] = i < (int)S.mat_bend.size() ? S.mat_bend[i] : 0.0;
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

ncpadj_status ncpadj_scene_refactor(ncpadj_scene scene, const double* E, const double* nu, void* stream) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(scene && E && nu, "NULL argument");
    NCPADJ_REQUIRE(scene->ctx, "scene without a context");
    NCPADJ_CUDA_TRY(cudaSetDevice(scene->ctx->c.device));
    Scene& S = scene->s;
    for (int t = 0; t < S.nt; ++t)
      NCPADJ_REQUIRE(E[t] > 0 && std::isfinite(E[t]) && nu[t] > -1.0 && nu[t] < 0.5,
                     "tet " + std::to_string(t) + ": need E > 0 and -1 < nu < 0.5");
    // work already queued on the stream may still read the arrays that are rebuilt
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    refactor_scene(S, E, nu, S.mat_bend.data());
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_scene_get_material(ncpadj_scene scene, double* E, double* nu) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(scene && E && nu, "NULL argument");
    const Scene& S = scene->s;
    std::copy(S.mat_E.begin(), S.mat_E.end(), E);
    std::copy(S.mat_nu.begin(), S.mat_nu.end(), nu);
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

void ncpadj_scene_destroy(ncpadj_scene s) {
  if (!s) return;
  if (s->s.flags_host) cudaFreeHost(s->s.flags_host);
  if (s->s.scal_host) cudaFreeHost(s->s.scal_host);
  if (s->s.gs_host) cudaFreeHost(s->s.gs_host);
  if (s->s.gs_inner_host) cudaFreeHost(s->s.gs_inner_host);
  if (s->s.gs_map_host) cudaFreeHost(s->s.gs_map_host);
  if (s->s.step_exec) cudaGraphExecDestroy(s->s.step_exec);
  if (s->s.bstep_exec) cudaGraphExecDestroy(s->s.bstep_exec);
  if (s->s.bmap_host) cudaFreeHost(s->s.bmap_host);
  if (s->s.btab_host) cudaFreeHost(s->s.btab_host);
  for (auto e : s->s.bev)
    if (e) cudaEventDestroy(e);
  for (auto e : s->s.gs_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : s->s.ev)
    if (e) cudaEventDestroy(e);
  delete s;
}

ncpadj_status ncpadj_scene_set_fibres(ncpadj_scene scene, const double* fibre) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(scene && fibre, "NULL argument");
    Scene& S = scene->s;
    NCPADJ_REQUIRE(S.nvpe == 4, "actuation fibres belong to tet scenes");
    for (int t = 0; t < S.nt; ++t) {
      const double* d = fibre + 3 * (size_t)t;
      const double n2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      NCPADJ_REQUIRE(std::isfinite(n2) && std::fabs(n2 - 1.0) <= 2e-6, "fibre " + std::to_string(t) + " is not a unit vector");
    }
    if (scene->ctx) NCPADJ_CUDA_TRY(cudaSetDevice(scene->ctx->c.device));
    S.fibre.ensure(sizeof(double) * 3 * (size_t)std::max(S.nt, 1));
    NCPADJ_CUDA_TRY(cudaMemcpy(S.fibre.p, fibre, sizeof(double) * 3 * (size_t)S.nt, cudaMemcpyHostToDevice));
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_scene_set_chunk(ncpadj_scene scene, int32_t entries) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(scene, "NULL scene");
    NCPADJ_REQUIRE(entries == 128 || entries == 256 || entries == 512, "entries must be 128, 256 or 512");
    Scene& S = scene->s;
    if (scene->ctx) NCPADJ_CUDA_TRY(cudaSetDevice(scene->ctx->c.device));
    if (entries != S.chunk) rechunk(S, entries);
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_scene_set_model(ncpadj_scene scene, const int32_t* model) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(scene, "NULL scene");
    Scene& S = scene->s;
    bool any = false;
    std::vector<int8_t> m8;
    if (model) {
      m8.resize((size_t)std::max(S.nt, 1), 0);
      for (int t = 0; t < S.nt; ++t) {
        NCPADJ_REQUIRE(model[t] >= NCPADJ_MODEL_NEO_HOOKEAN && model[t] <= NCPADJ_MODEL_ARAP,
                       "model " + std::to_string(model[t]) + " of tet " + std::to_string(t) + " is not a NCPADJ_MODEL_*");
        m8[t] = (int8_t)model[t];
        any = any || model[t] != NCPADJ_MODEL_NEO_HOOKEAN;
      }
    }
    if (scene->ctx) NCPADJ_CUDA_TRY(cudaSetDevice(scene->ctx->c.device));
    if (any) {
      S.model.ensure(m8.size());
      NCPADJ_CUDA_TRY(cudaMemcpy(S.model.p, m8.data(), m8.size(), cudaMemcpyHostToDevice));
    }
    S.model_any = any;
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_scene_get_info(ncpadj_scene s, ncpadj_scene_info* out) {
  if (!s || !out) {
    set_error("NULL argument");
    return NCPADJ_ERR_INVALID_ARG;
  }
  out->n_verts = s->s.nv;
  out->n_tets = s->s.nt;
  out->n_blocks = s->s.nb;
  out->nnz_L = s->s.nnz_L;
  out->nnz_Linv = s->s.nnz_S;
  out->ms_factor = s->s.ms_factor;
  out->n_scenes = s->s.n_scenes;
  out->element_verts = s->s.nvpe;
  out->n_hinges = s->s.n_bend;
  return NCPADJ_OK;
}

ncpadj_status ncpadj_elastic_solve(ncpadj_ctx ctx, ncpadj_scene scene, const double* x, double* y, void* stream) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(ctx && scene && x && y && x != y, "NULL or aliased argument");
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    Scene& S = scene->s;
    cudaStream_t st = (cudaStream_t)stream;
    S.io.ensure(sizeof(double) * 3 * (size_t)S.nv);
    SinvArgs a{S.nv, S.S_ptr.as<int64_t>(), S.S_c0.as<int32_t>(), S.S_val.as<double>(), S.St_ptr.as<int64_t>(),
               S.St_col.as<int32_t>(), S.St_val.as<double>(), S.perm.as<int32_t>(), S.nS_chunks, S.nSt_chunks,
               S.S_crow.as<int32_t>(), S.St_crow.as<int32_t>(), S.S_cbeg.as<int64_t>(), S.S_cend.as<int64_t>(),
               S.St_cbeg.as<int64_t>(), S.St_cend.as<int64_t>()};
    a.chunk = S.chunk;
    S.xpos.ensure(sizeof(double) * 3 * (size_t)S.nv + 64);
    a.xpos = S.xpos.as<double>();
    launch_ainv(a, x, S.io.as<double>(), y, st);
    NCPADJ_CUDA_TRY(cudaGetLastError());
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_elastic_solve_mixed(ncpadj_ctx ctx, ncpadj_scene scene, const double* x, double* y,
                                         void* stream) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(ctx && scene && x && y && x != y, "NULL or aliased argument");
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    Scene& S = scene->s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n3 = 3 * (size_t)S.nv;
    S.io.ensure(sizeof(float) * n3 + 64);
    SinvArgs a{S.nv, S.S_ptr.as<int64_t>(), S.S_c0.as<int32_t>(), S.S_val.as<double>(), S.St_ptr.as<int64_t>(),
               S.St_col.as<int32_t>(), S.St_val.as<double>(), S.perm.as<int32_t>(), S.nS_chunks, S.nSt_chunks,
               S.S_crow.as<int32_t>(), S.St_crow.as<int32_t>(), S.S_cbeg.as<int64_t>(), S.S_cend.as<int64_t>(),
               S.St_cbeg.as<int64_t>(), S.St_cend.as<int64_t>(), S.S_val32.as<float>(), S.St_val32.as<float>()};
    a.chunk = S.chunk;
    S.xpos.ensure(sizeof(double) * n3 + sizeof(float) * n3 + 64);
    a.xpos = S.xpos.as<double>();
    a.xpos32 = reinterpret_cast<float*>(S.xpos.as<double>() + n3);
    launch_ainv32(a, x, nullptr, S.io.as<float>(), y, st);
    NCPADJ_CUDA_TRY(cudaGetLastError());
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_dense_inverse(ncpadj_ctx ctx, int32_t n, const double* C, double* Cinv, int32_t precision,
                                   void* stream) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(ctx && C && Cinv && C != Cinv, "NULL or aliased argument");
    NCPADJ_REQUIRE(n > 0 && n <= gj_cols_max_dim(), "n out of range");
    NCPADJ_REQUIRE(precision == NCPADJ_FP64 || precision == NCPADJ_MIXED || precision == NCPADJ_TF32X3,
                   "bad precision");
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    cudaStream_t st = (cudaStream_t)stream;
    Ctx& X = ctx->c;
    if (precision == NCPADJ_TF32X3) {
      const size_t ne = (size_t)n * n;
      X.inv_mat.ensure(sizeof(float) * ne + sizeof(int32_t) * (size_t)n + sizeof(int) * FLAG_COUNT + 256);
      // its own scratch: the Gauss-Jordan inverse keeps sync words at the start of inv_work that must stay zero
      X.rec_work.ensure(bgj_scratch_bytes(n));
      float* B = X.inv_mat.as<float>();
      int32_t* piv = reinterpret_cast<int32_t*>(B + ne);
      int* flags = reinterpret_cast<int*>(piv + n);
      NCPADJ_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * FLAG_COUNT, st));
      launch_convert_f32((long)ne, C, B, st);
      if (!launch_bgj_inverse(n, B, n, X.rec_work.p, piv, flags, X.sm_count, st)) {
        cudaGetLastError();
        throw Error{NCPADJ_ERR_UNSUPPORTED, "the cooperative grid of the tensor-core inverse does not fit"};
      }
      NCPADJ_CUDA_TRY(cudaGetLastError());
      int fh[FLAG_COUNT];
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(fh, flags, sizeof(fh), cudaMemcpyDeviceToHost, st));
      NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
      if (fh[FLAG_TIMEOUT]) throw Error{NCPADJ_ERR_TIMEOUT, "a wait of the tensor-core inverse timed out"};
      if (fh[FLAG_SINGULAR]) throw Error{NCPADJ_ERR_NONFINITE, "a diagonal block is singular"};
      launch_unpermute_inverse(n, B, true, piv, Cinv, st);
      NCPADJ_CUDA_TRY(cudaGetLastError());
      return NCPADJ_OK;
    }
    const bool fp32 = precision == NCPADJ_MIXED;
    const size_t ne = (size_t)n * n;
    const size_t mat_bytes = (fp32 ? sizeof(float) : sizeof(double)) * ne + sizeof(int32_t) * (size_t)n +
                             sizeof(int) * FLAG_COUNT + 256;
    X.inv_mat.ensure(mat_bytes);
    const size_t wbytes = gj_cols_scratch_bytes(n, fp32);
    if (X.inv_work.bytes < wbytes) {
      X.inv_work.ensure(wbytes);
      NCPADJ_CUDA_TRY(cudaMemset(X.inv_work.p, 0, wbytes));
    }
    char* base = X.inv_mat.as<char>();
    void* B = base;
    int32_t* piv = reinterpret_cast<int32_t*>(base + (fp32 ? sizeof(float) : sizeof(double)) * ne);
    int* flags = reinterpret_cast<int*>(piv + n);
    NCPADJ_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * FLAG_COUNT, st));
    bool ok;
    if (fp32) {
      launch_convert_f32((long)ne, C, static_cast<float*>(B), st);
      ok = launch_gj_cols32(n, static_cast<float*>(B), X.inv_work.p, piv, flags, X.sm_count, st);
    } else {
      NCPADJ_CUDA_TRY(cudaMemcpyAsync(B, C, sizeof(double) * ne, cudaMemcpyDeviceToDevice, st));
      ok = launch_gj_cols64(n, static_cast<double*>(B), X.inv_work.p, piv, flags, X.sm_count, st);
    }
    if (!ok) {
      cudaGetLastError();
      throw Error{NCPADJ_ERR_UNSUPPORTED, "the dense inverse could not be launched for n = " + std::to_string(n)};
    }
    int fh[FLAG_COUNT];
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(fh, flags, sizeof(fh), cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    if (fh[FLAG_TIMEOUT]) throw Error{NCPADJ_ERR_TIMEOUT, "a wait of the dense inverse timed out"};
    if (fh[FLAG_SINGULAR]) throw Error{NCPADJ_ERR_NONFINITE, "the matrix is singular"};
    launch_unpermute_inverse(n, B, fp32, piv, Cinv, st);
    NCPADJ_CUDA_TRY(cudaGetLastError());
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_dense_gemm(ncpadj_ctx ctx, int32_t M, int32_t N, int32_t K, float alpha, const float* A,
                                int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                                int32_t split, void* stream) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(ctx && A && B && C, "NULL argument");
    NCPADJ_REQUIRE(M >= 1 && N >= 1 && K >= 1, "M, N and K must be positive");
    NCPADJ_REQUIRE(lda >= K && ldb >= N && ldc >= N, "a leading dimension is below its row length");
    NCPADJ_REQUIRE(split == 0 || split == 1, "split must be 0 or 1");
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    cudaStream_t st = (cudaStream_t)stream;
    Ctx& X = ctx->c;
    X.gemm_flags.ensure(sizeof(int) * FLAG_COUNT);
    int* flags = X.gemm_flags.as<int>();
    NCPADJ_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * FLAG_COUNT, st));
    launch_tc_gemm(GemmArgs{M, N, K, alpha, beta, A, (long)lda, B, (long)ldb, C, (long)ldc, split, flags}, st);
    NCPADJ_CUDA_TRY(cudaGetLastError());
    int fh[FLAG_COUNT];
    NCPADJ_CUDA_TRY(cudaMemcpyAsync(fh, flags, sizeof(fh), cudaMemcpyDeviceToHost, st));
    NCPADJ_CUDA_TRY(cudaStreamSynchronize(st));
    if (fh[FLAG_TIMEOUT]) throw Error{NCPADJ_ERR_TIMEOUT, "a wait of the tensor-core inverse timed out"};
    return NCPADJ_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_forward_step(ncpadj_ctx ctx, ncpadj_scene scene, const ncpadj_contacts* contacts,
                                  const ncpadj_forward_input* input, const ncpadj_options* opt, double newton_tol,
                                  int32_t max_newton, double* q_out, double* lambda_out, ncpadj_forward_stats* stats,
                                  void* stream) {
  g_last_error.clear();
  try {
    if (ctx) NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    return forward_step(ctx, scene, contacts, input, opt, newton_tol, max_newton, q_out, lambda_out, stats,
                        (cudaStream_t)stream);
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_adjoint_batch(ncpadj_ctx ctx, ncpadj_scene batch, int32_t n_scenes,
                                   const ncpadj_contacts* contacts, const ncpadj_state* states,
                                   const ncpadj_seed* seeds, const ncpadj_options* opt, ncpadj_grads* grads,
                                   ncpadj_stats* stats, void* stream) {
  g_last_error.clear();
  try {
    NCPADJ_REQUIRE(ctx && batch, "NULL context or scene");
    NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    return adjoint_batch(ctx, batch, n_scenes, contacts, states, seeds, opt, grads, stats,
                         static_cast<cudaStream_t>(stream));
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

ncpadj_status ncpadj_adjoint_step(ncpadj_ctx ctx, ncpadj_scene scene, const ncpadj_contacts* contacts,
                                  const ncpadj_state* state, const ncpadj_seed* seed, const ncpadj_options* opt,
                                  ncpadj_grads* grads, ncpadj_stats* stats, void* stream) {
  g_last_error.clear();
  try {
    if (ctx) NCPADJ_CUDA_TRY(cudaSetDevice(ctx->c.device));
    return adjoint_step(ctx, scene, contacts, state, seed, opt, grads, stats, (cudaStream_t)stream);
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail(Error{NCPADJ_ERR_OOM, e.what()});
  }
}

}  // extern "C"
