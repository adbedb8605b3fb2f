// Per-tet and per-contact kernels of the adjoint step.
//
//  * tet_assemble: F = D_s D_m^{-1}; signed SVD of F; Neo-Hookean singular-value prox
//    theta(sigma) and its derivatives W = dtheta/dsigma, dtheta/dmu, dtheta/dlambda
//    (App. B.2, B.3); the projection Jacobian dvecP/dvecF in its SVD closed form
//    (Sec. 4.3, App. B.0, with the T term carrying N) folded directly into the 10 unique
//    3x3 blocks of h^2 w_i G_i^T (I - dP/dF) G_i, added into the fixed block pattern of
//    script_A (Sec. 4.4, matrix assembly); and the per-tet tensors used later by the
//    material-parameter contractions (App. B.3).
//  * contact_blocks: the smoothed-FB contact Jacobian K_c = R^T Khat R and k_mu
//    (Eq. final_diff_contact, App. A.1), added as h^2 F^T K_c^T F into the vertex's
//    diagonal block (the matrix held is script_A^T).
//  * contractions: dL/dx = z^T K_x (Eq. compute_gradient, App. B.3).
#include <math.h>

#include "kernels.cuh"

namespace ncpadj {
namespace {

template <typename T> struct Num;
template <> struct Num<double> {
  static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
  static __device__ __forceinline__ double lg(double x) { return log(x); }
  static constexpr double tol_eig = 1e-30;   // relative off-diagonal^2 of the Jacobi sweeps
  static constexpr double tol_newton = 1e-14;
  static constexpr int sweeps = 12;
};
template <> struct Num<float> {
  static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float lg(float x) { return logf(x); }
  static constexpr float tol_eig = 1e-14f;
  static constexpr float tol_newton = 2e-6f;
  static constexpr int sweeps = 8;
};

// One Jacobi rotation zeroing a[p][q] of a symmetric 3x3 matrix; v accumulates the rotations
// (symmetric Schur decomposition, Golub & Van Loan Sec. 8.5).
template <typename T>
__device__ __forceinline__ void jacobi_rotate(T a[3][3], T v[3][3], int p, int q) {
  T apq = a[p][q];
  if (apq == T(0)) return;
  T tau = (a[q][q] - a[p][p]) / (T(2) * apq);
  T t;
  if (fabs(tau) > T(1e15)) t = T(0.5) / tau;
  else t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + Num<T>::sq(tau * tau + T(1)));
  T c = T(1) / Num<T>::sq(t * t + T(1));
  T s = t * c;
  a[p][p] -= t * apq;
  a[q][q] += t * apq;
  a[p][q] = a[q][p] = T(0);
  int r = 3 - p - q;
  T arp = a[r][p], arq = a[r][q];
  a[r][p] = a[p][r] = c * arp - s * arq;
  a[r][q] = a[q][r] = s * arp + c * arq;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T vkp = v[k][p], vkq = v[k][q];
    v[k][p] = c * vkp - s * vkq;
    v[k][q] = s * vkp + c * vkq;
  }
}

// Signed SVD F = U diag(sig) V^T with det U = det V = +1: eigenvectors V of F^T F by cyclic
// Jacobi, sorted by decreasing singular value, then U from F V by Gram-Schmidt with
// u_3 = u_1 x u_2 (so that the sign of det F lands on sig_3).  Returns false if F is
// singular or inverted (sig_3 <= 0).
template <typename T>
__device__ bool svd3(const T F[3][3], T U[3][3], T sig[3], T V[3][3]) {
  T a[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) a[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? T(1) : T(0);
  for (int sw = 0; sw < Num<T>::sweeps; ++sw) {
    T off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    T dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= Num<T>::tol_eig * dg) break;
    jacobi_rotate(a, V, 0, 1);
    jacobi_rotate(a, V, 0, 2);
    jacobi_rotate(a, V, 1, 2);
  }
  T ev[3] = {a[0][0], a[1][1], a[2][2]};
  // sort decreasing (swap V columns along)
#pragma unroll
  for (int pass = 0; pass < 2; ++pass)
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (ev[i] < ev[i + 1]) {
        T tmp = ev[i]; ev[i] = ev[i + 1]; ev[i + 1] = tmp;
#pragma unroll
        for (int k = 0; k < 3; ++k) { T t2 = V[k][i]; V[k][i] = V[k][i + 1]; V[k][i + 1] = t2; }
      }
  T detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
           V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  if (detV < T(0))
#pragma unroll
    for (int k = 0; k < 3; ++k) V[k][2] = -V[k][2];
  T f[3][3];  // columns F v_i
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int r = 0; r < 3; ++r) f[i][r] = F[r][0] * V[0][i] + F[r][1] * V[1][i] + F[r][2] * V[2][i];
  T n0 = Num<T>::sq(f[0][0] * f[0][0] + f[0][1] * f[0][1] + f[0][2] * f[0][2]);
  if (!(n0 > T(0))) return false;
  T u0[3] = {f[0][0] / n0, f[0][1] / n0, f[0][2] / n0};
  T d = u0[0] * f[1][0] + u0[1] * f[1][1] + u0[2] * f[1][2];
  T w1[3] = {f[1][0] - d * u0[0], f[1][1] - d * u0[1], f[1][2] - d * u0[2]};
  T n1 = Num<T>::sq(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
  if (!(n1 > T(0))) return false;
  T u1[3] = {w1[0] / n1, w1[1] / n1, w1[2] / n1};
  T u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
  T s2 = u2[0] * f[2][0] + u2[1] * f[2][1] + u2[2] * f[2][2];
  sig[0] = n0;
  sig[1] = n1;
  sig[2] = s2;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    U[r][0] = u0[r];
    U[r][1] = u1[r];
    U[r][2] = u2[r];
  }
  return s2 > T(0);
}

// Neo-Hookean prox on the singular values (App. B.2): solve
//   g(theta) = mu (3 theta - 2 sigma - 1/theta) + lambda log(J) / theta = 0,  J = prod theta,
// by damped Newton from theta = sigma; dg/dtheta = Dg + lambda a a^T, Dg = 3 mu + (mu - lambda log J) a^2,
// a = 1/theta, inverted by Sherman-Morrison.  Outputs theta, Hinv = (dg/dtheta)^{-1} (symmetric),
// log J.
template <typename T>
__device__ void nh_prox(const T sig[3], T mu, T lam, T th[3], T Hinv[3][3], T& logJ) {
  th[0] = sig[0]; th[1] = sig[1]; th[2] = sig[2];
  T a[3], Dg[3];
  for (int it = 0; it < 40; ++it) {
    logJ = Num<T>::lg(th[0] * th[1] * th[2]);
    T g[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a[i] = T(1) / th[i];
      g[i] = mu * (T(3) * th[i] - T(2) * sig[i] - a[i]) + lam * logJ * a[i];
    }
    T gmax = fmax(fabs(g[0]), fmax(fabs(g[1]), fabs(g[2])));
    if (gmax <= Num<T>::tol_newton * mu) break;
    T Dia[3], Dig[3], aDa = 0, aDg = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Dg[i] = T(3) * mu + (mu - lam * logJ) * a[i] * a[i];
      Dia[i] = a[i] / Dg[i];
      Dig[i] = g[i] / Dg[i];
      aDa += a[i] * Dia[i];
      aDg += a[i] * Dig[i];
    }
    T coef = lam * aDg / (T(1) + lam * aDa);
    T step[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) step[i] = -(Dig[i] - coef * Dia[i]);
    T t = T(1);
    for (int k = 0; k < 30; ++k) {
      if (th[0] + t * step[0] > T(0) && th[1] + t * step[1] > T(0) && th[2] + t * step[2] > T(0)) break;
      t *= T(0.5);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) th[i] += t * step[i];
  }
  logJ = Num<T>::lg(th[0] * th[1] * th[2]);
  T Dia[3], aDa = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    a[i] = T(1) / th[i];
    Dg[i] = T(3) * mu + (mu - lam * logJ) * a[i] * a[i];
    Dia[i] = a[i] / Dg[i];
    aDa += a[i] * Dia[i];
  }
  T c = lam / (T(1) + lam * aDa);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Hinv[i][j] = ((i == j) ? T(1) / Dg[i] : T(0)) - c * Dia[i] * Dia[j];
}

// The local projection on the singular values for the three isotropic models of App. B.2, with
// what the Jacobian and the contractions need: theta, W = dtheta/dsigma, the total dtheta/dmu and
// dtheta/dlambda of App. B.3 (w = 2 mu varies with mu), and the divided differences
// Ad[i][j] = (theta_i - theta_j)/(sigma_i - sigma_j) in a form without cancellation.
//  - Neo-Hookean: Newton on its stationarity condition (nh_prox); subtracting the conditions of
//    components i and j gives Ad[i][j] = 2 mu / (3 mu + (mu - lambda log J) / (theta_i theta_j)),
//    which also covers the degenerate limit of App. B.4.
//  - co-rotational: the condition 4 mu (theta - 1) + lambda tr(theta - 1) 1 = 2 mu (sigma - 1) is
//    linear, so theta - 1 = W (sigma - 1) with the constant W = I/2 - c 1 1^T,
//    c = lambda / (2 (4 mu + 3 lambda)); Ad = 1/2.
//  - ARAP: theta = 1, W = 0, no parameter dependence (mu acts only through w); Ad = 0.
template <typename T>
__device__ void local_prox(int model, const T sig[3], T mu, T lam, T th[3], T W[3][3], T dmu[3], T dlam[3],
                           T Ad[3][3]) {
  if (model == MODEL_COROTATIONAL) {
    const T den = T(4) * mu + T(3) * lam;
    const T c = lam / (T(2) * den);
    const T s = (sig[0] - T(1)) + (sig[1] - T(1)) + (sig[2] - T(1));
    const T gm = T(2) * lam * s / (den * den), gl = -T(2) * mu * s / (den * den);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      th[i] = T(0.5) * (sig[i] + T(1)) - c * s;
      dmu[i] = gm;
      dlam[i] = gl;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        W[i][j] = (i == j ? T(0.5) : T(0)) - c;
        Ad[i][j] = T(0.5);
      }
    }
    return;
  }
  if (model == MODEL_ARAP) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      th[i] = T(1);
      dmu[i] = dlam[i] = T(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) W[i][j] = Ad[i][j] = T(0);
    }
    return;
  }
  T Hinv[3][3], logJ;
  nh_prox<T>(sig, mu, lam, th, Hinv, logJ);
  // W = 2 mu Hinv ; dtheta/dmu = -Hinv (3 theta - 2 sigma - 1/theta) ; dtheta/dlam = -Hinv (log J / theta)
  T gm[3], gl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gm[i] = T(3) * th[i] - T(2) * sig[i] - T(1) / th[i];
    gl[i] = logJ / th[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dmu[i] = -(Hinv[i][0] * gm[0] + Hinv[i][1] * gm[1] + Hinv[i][2] * gm[2]);
    dlam[i] = -(Hinv[i][0] * gl[0] + Hinv[i][1] * gl[1] + Hinv[i][2] * gl[2]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      W[i][j] = T(2) * mu * Hinv[i][j];
      Ad[i][j] = (i == j) ? T(0) : T(2) * mu / (T(3) * mu + (mu - lam * logJ) / (th[i] * th[j]));
    }
  }
}

// theta alone (the forward residual)
template <typename T>
__device__ void local_theta(int model, const T sig[3], T mu, T lam, T th[3]) {
  if (model == MODEL_COROTATIONAL) {
    const T c = lam / (T(2) * (T(4) * mu + T(3) * lam));
    const T s = (sig[0] - T(1)) + (sig[1] - T(1)) + (sig[2] - T(1));
#pragma unroll
    for (int i = 0; i < 3; ++i) th[i] = T(0.5) * (sig[i] + T(1)) - c * s;
  } else if (model == MODEL_ARAP) {
    th[0] = th[1] = th[2] = T(1);
  } else {
    T Hinv[3][3], logJ;
    nh_prox<T>(sig, mu, lam, th, Hinv, logJ);
  }
}

template <typename T>
__device__ __forceinline__ void atomic_add_out(double* p, T v) { atomicAdd(p, (double)v); }
template <typename T>
__device__ __forceinline__ void atomic_add_out(float* p, T v) { atomicAdd(p, (float)v); }

template <typename T, typename OutT>
__global__ void __launch_bounds__(128) k_tet_assemble(TetArgs A, OutT* bsr) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.nt) return;
  int vid[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) vid[a] = A.tets[4 * t + a];
  T g[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) g[a][k] = (T)A.gvec[12 * t + 3 * a + k];
  // F = sum_a x_a g_a^T
  T F[3][3] = {};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double x0 = A.q[3 * vid[a]], x1 = A.q[3 * vid[a] + 1], x2 = A.q[3 * vid[a] + 2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      F[0][k] += (T)x0 * g[a][k];
      F[1][k] += (T)x1 * g[a][k];
      F[2][k] += (T)x2 * g[a][k];
    }
  }
  T U[3][3], V[3][3], sig[3];
  if (!svd3<T>(F, U, sig, V)) {
    atomicExch(&A.flags[FLAG_INVERTED], 1);
    return;
  }
  const T mu = (T)A.mu[t], lam = (T)A.lam[t];
  T th[3], W[3][3], dmu[3], dlam[3], Ad[3][3];
  local_prox<T>(A.model ? A.model[t] : MODEL_NEO_HOOKEAN, sig, mu, lam, th, W, dmu, dlam, Ad);
  // off-diagonal coefficients M_ij = (A_ij + B_ij)/2, N_ij = (A_ij - B_ij)/2 (App. B.0), with the
  // divided difference A_ij from local_prox
  T Mc[3][3], Nc[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (i == j) { Mc[i][j] = Nc[i][j] = T(0); continue; }
      T Aij = Ad[i][j];
      T Bij = (th[i] + th[j]) / (sig[i] + sig[j]);
      Mc[i][j] = T(0.5) * (Aij + Bij);
      Nc[i][j] = T(0.5) * (Aij - Bij);
    }
  // c_i[a] = g_a . v_i
  T c[3][4];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 4; ++a) c[i][a] = g[a][0] * V[0][i] + g[a][1] * V[1][i] + g[a][2] * V[2][i];
  const T hw = (T)(A.h * A.h) * T(2) * mu * (T)A.vol[t];
  if (bsr != nullptr) {
  // blocks (a, b), a <= b:  U Q U^T with, in the U basis,
  //   Q_pp = g_a.g_b - W_pp c_p[a] c_p[b] - sum_{j != p} M_pj c_j[a] c_j[b]
  //   Q_pq = -W_pq c_p[a] c_q[b] - N_pq c_q[a] c_p[b]          (p != q)
#pragma unroll 1
  for (int a = 0; a < 4; ++a) {
#pragma unroll 1
    for (int b = a; b < 4; ++b) {
      T gg = c[0][a] * c[0][b] + c[1][a] * c[1][b] + c[2][a] * c[2][b];
      T Q[3][3];
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int qq = 0; qq < 3; ++qq) {
          if (p == qq) {
            T s = gg - W[p][p] * c[p][a] * c[p][b];
#pragma unroll
            for (int j = 0; j < 3; ++j)
              if (j != p) s -= Mc[p][j] * c[j][a] * c[j][b];
            Q[p][qq] = s;
          } else {
            Q[p][qq] = -W[p][qq] * c[p][a] * c[qq][b] - Nc[p][qq] * c[qq][a] * c[p][b];
          }
        }
      T UQ[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int qq = 0; qq < 3; ++qq) UQ[r][qq] = U[r][0] * Q[0][qq] + U[r][1] * Q[1][qq] + U[r][2] * Q[2][qq];
      T blk[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) blk[r][s] = hw * (UQ[r][0] * U[s][0] + UQ[r][1] * U[s][1] + UQ[r][2] * U[s][2]);
      OutT* dst = bsr + 9 * (size_t)A.slot[16 * t + 4 * a + b];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) atomic_add_out(dst + 3 * r + s, blk[r][s]);
      if (a != b) {
        OutT* dst2 = bsr + 9 * (size_t)A.slot[16 * t + 4 * b + a];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int s = 0; s < 3; ++s) atomic_add_out(dst2 + 3 * r + s, blk[s][r]);
      }
    }
  }
  }
  if (A.tetdata == nullptr) return;
  // contraction tensors P_mu = U diag(e_mu) V^T, P_lam = U diag(e_lam) V^T with
  // e_mu = 2 h^2 V (mu dtheta/dmu + theta - sigma), e_lam = 2 h^2 V mu dtheta/dlambda
  const double h2v2 = 2.0 * A.h * A.h * A.vol[t];
  double em[3], el[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    em[i] = h2v2 * ((double)mu * dmu[i] + (double)th[i] - (double)sig[i]);
    el[i] = h2v2 * (double)mu * dlam[i];
  }
  double* td = A.tetdata + 18 * (size_t)t;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      double um = 0, ul = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double uv = (double)U[r][i] * (double)V[s][i];
        um += em[i] * uv;
        ul += el[i] * uv;
      }
      td[3 * r + s] = um;
      td[9 + 3 * r + s] = ul;
    }
}

// stable FB partials (1 - x/r, 1 - y/r), r = sqrt(x^2 + y^2 + 2 eps^2)
__device__ __forceinline__ void fb_partials(double x, double y, double e2, double& a, double& b) {
  double r = sqrt(x * x + y * y + e2);
  a = (y * y + e2) / (r * (r + x));
  b = (x * x + e2) / (r * (r + y));
}

template <typename OutT>
__global__ void k_contact_blocks(ContactArgs A, OutT* bsr) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.nc) return;
  const int v = A.vertex[c];
  double F[3][3];
#pragma unroll
  for (int i = 0; i < 9; ++i) F[i / 3][i % 3] = A.frame[9 * c + i];
  double qv[3], dq[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    qv[r] = A.q[3 * v + r];
    dq[r] = qv[r] - A.q_prev[3 * v + r];
  }
  const double dn = F[0][0] * qv[0] + F[0][1] * qv[1] + F[0][2] * qv[2] - A.d_n[c];
  double df1 = F[1][0] * dq[0] + F[1][1] * dq[1] + F[1][2] * dq[2];
  double df2 = F[2][0] * dq[0] + F[2][1] * dq[1] + F[2][2] * dq[2];
  if (A.d_f) {
    df1 -= A.d_f[2 * c];
    df2 -= A.d_f[2 * c + 1];
  }
  const double lam_n = A.lambda[3 * c], lf1 = A.lambda[3 * c + 1], lf2 = A.lambda[3 * c + 2];
  const double mu = A.mu[c];
  const double e2 = 2.0 * A.eps * A.eps;
  double an, bn;
  fb_partials(dn, lam_n, e2, an, bn);
  const double k11 = an / bn;
  double K[3][3] = {{k11, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double kmu[3] = {0, 0, 0};
  if (mu > 0.0) {
    const double s = sqrt(df1 * df1 + df2 * df2);
    double t1, t2, gam, k33;
    if (s > 0.0) {
      t1 = df1 / s;
      t2 = df2 / s;
      gam = -(lf1 * t1 + lf2 * t2);
      k33 = gam / s;
    } else {
      // no slip: the frame falls back on the force direction (App. A.1), no direction stiffness
      const double lf = sqrt(lf1 * lf1 + lf2 * lf2);
      if (lf > 0.0) { t1 = -lf1 / lf; t2 = -lf2 / lf; gam = lf; }
      else { t1 = 1.0; t2 = 0.0; gam = 0.0; atomicExch(&A.flags[FLAG_DOMAIN], 1); }
      k33 = 0.0;
    }
    double af, bf;
    fb_partials(s, mu * lam_n - gam, e2, af, bf);
    const double k22 = af / bf;
    // Khat = [[k11, 0, 0], [-mu k11, k22, 0], [0, 0, k33]],  R = [[1,0,0],[0,t1,t2],[0,-t2,t1]],  K = R^T Khat R
    double R[3][3] = {{1, 0, 0}, {0, t1, t2}, {0, -t2, t1}};
    double Kh[3][3] = {{k11, 0, 0}, {-mu * k11, k22, 0}, {0, 0, k33}};
    double KR[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) KR[i][j] = Kh[i][0] * R[0][j] + Kh[i][1] * R[1][j] + Kh[i][2] * R[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) K[i][j] = R[0][i] * KR[0][j] + R[1][i] * KR[1][j] + R[2][i] * KR[2][j];
    kmu[1] = lam_n * t1;  // R^T (0, lambda_n, 0)
    kmu[2] = lam_n * t2;
  }
  double* cd = A.cdata + 12 * (size_t)c;
#pragma unroll
  for (int i = 0; i < 9; ++i) cd[i] = K[i / 3][i % 3];
  cd[9] = kmu[0];
  cd[10] = kmu[1];
  cd[11] = kmu[2];
  // h^2 F^T K^T F (adjoint, script_A^T) or h^2 F^T K F (Newton matrix) into the diagonal block of v
  const double h2 = A.h * A.h;
  double KtF[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      KtF[i][j] = A.transpose ? K[0][i] * F[0][j] + K[1][i] * F[1][j] + K[2][i] * F[2][j]
                              : K[i][0] * F[0][j] + K[i][1] * F[1][j] + K[i][2] * F[2][j];
  OutT* dst = bsr + 9 * (size_t)A.diag_slot[v];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      double w = F[0][r] * KtF[0][s] + F[1][r] * KtF[1][s] + F[2][r] * KtF[2][s];
      atomicAdd(dst + 3 * r + s, (OutT)(h2 * w));
    }
}

template <typename OutT>
__global__ void k_bsr_init(int nv, int nb, const int32_t* diag_slot, const double* mass, OutT* bsr) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < 9L * nb) bsr[i] = OutT(0);
}
template <typename OutT>
__global__ void k_bsr_mass(int nv, const int32_t* diag_slot, const double* mass, OutT* bsr) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  OutT* d = bsr + 9 * (size_t)diag_slot[v];
  d[0] = d[4] = d[8] = (OutT)mass[v];
}

__global__ void k_contract_vertex(ContractArgs A) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * A.nv) return;
  const double z = A.z[i], m = A.mass[i / 3];
  if (A.dL_dq_prev) A.dL_dq_prev[i] = m * z - (A.dL_dv ? A.dL_dv[i] / A.h : 0.0);
  if (A.dL_dv_prev) A.dL_dv_prev[i] = A.h * m * z;
  if (A.dL_dfext) A.dL_dfext[i] = A.h * A.h * z;
}

// contact parts: dL/dqbar += h^2 F^T P_f K^T F z_v ; dL/dmu_c = -h^2 (F z_v) . k_mu
__global__ void k_contract_contact(ContractArgs A) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.nc) return;
  const int v = A.cvertex[c];
  const double* F = A.frame + 9 * (size_t)c;
  const double* cd = A.cdata + 12 * (size_t)c;
  const double zv[3] = {A.z[3 * v], A.z[3 * v + 1], A.z[3 * v + 2]};
  double y[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = F[3 * i] * zv[0] + F[3 * i + 1] * zv[1] + F[3 * i + 2] * zv[2];
  const double h2 = A.h * A.h;
  if (A.dL_dq_prev) {
    double w[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) w[j] = cd[j] * y[0] + cd[3 + j] * y[1] + cd[6 + j] * y[2];  // K^T y
    w[0] = 0.0;                                                                           // P_f
#pragma unroll
    for (int r = 0; r < 3; ++r)
      atomicAdd(&A.dL_dq_prev[3 * v + r], h2 * (F[r] * w[0] + F[3 + r] * w[1] + F[6 + r] * w[2]));
  }
  const double g = -h2 * (y[0] * cd[9] + y[1] * cd[10] + y[2] * cd[11]);
  if (A.dL_dmu_contact) A.dL_dmu_contact[c] = g;
  if (A.dL_dmu) atomicAdd(&A.dL_dmu[A.region ? A.region[c] : 0], g);
}

__global__ void k_contract_tet(ContractArgs A) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.nt) return;
  const double* td = A.tetdata + 18 * (size_t)t;
  const double* g = A.gvec + 12 * (size_t)t;
  double dmu = 0, dlam = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int v = A.tets[4 * t + a];
    const double za[3] = {A.z[3 * v], A.z[3 * v + 1], A.z[3 * v + 2]};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double pm = td[3 * r] * g[3 * a] + td[3 * r + 1] * g[3 * a + 1] + td[3 * r + 2] * g[3 * a + 2];
      double pl = td[9 + 3 * r] * g[3 * a] + td[9 + 3 * r + 1] * g[3 * a + 1] + td[9 + 3 * r + 2] * g[3 * a + 2];
      dmu += za[r] * pm;
      dlam += za[r] * pl;
    }
  }
  const double* ld = A.lame_d + 4 * (size_t)t;
  if (A.dL_dE) A.dL_dE[t] = dmu * ld[0] + dlam * ld[1];
  if (A.dL_dnu) A.dL_dnu[t] = dmu * ld[2] + dlam * ld[3];
}

__global__ void k_check_contacts(int nc, const int32_t* vertex, const int32_t* region, int nv, int nreg, int* flags) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int v = vertex[c];
  bool bad = v < 0 || v >= nv;
  if (region) bad = bad || region[c] < 0 || region[c] >= nreg;
  if (bad) atomicExch(&flags[FLAG_BADINDEX], 1);
}

// ---- bilateral bindings on single vertices (Eq. binding): phi_b = q_v - d_b + E_b lambda_b = 0 ----

// a binding vertex out of range or a compliance that is not a positive finite number
__global__ void k_check_bindings(int nb, const int32_t* vertex, const double* compliance, int nv, int* flags) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int v = vertex[b];
  const double e = compliance[b];
  if (v < 0 || v >= nv || !(e > 0.0) || !isfinite(e)) atomicExch(&flags[FLAG_BADINDEX], 1);
}
// h^2 J_b^T E_b^{-1} J_b = h^2 / E_b I_3 on the bound vertex's diagonal block (Eq. differential_2)
template <typename OutT>
__global__ void k_binding_blocks(int nb, const int32_t* __restrict__ vertex, const double* __restrict__ compliance,
                                 const int32_t* __restrict__ diag_slot, double h, OutT* bsr) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double k = h * h / compliance[b];
  OutT* dst = bsr + 9 * (size_t)diag_slot[vertex[b]];
  atomic_add_out(dst + 0, k);
  atomic_add_out(dst + 4, k);
  atomic_add_out(dst + 8, k);
}
// the binding force in the momentum residual: -h^2 J_b^T lambda_b = h^2 (q_v - d_b) / E_b at v
__global__ void k_binding_force(int nb, const int32_t* __restrict__ vertex, const double* __restrict__ target,
                                const double* __restrict__ compliance, const double* __restrict__ q, double h,
                                double* R) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int v = vertex[b];
  const double k = h * h / compliance[b];
#pragma unroll
  for (int r = 0; r < 3; ++r) atomicAdd(&R[3 * (size_t)v + r], k * (q[3 * (size_t)v + r] - target[3 * (size_t)b + r]));
}
// dL/dd_b = h^2 z_v / E_b ; dL/dE_b = h^2 z_v . (q_v - d_b) / E_b^2 (Eq. compute_gradient)
__global__ void k_binding_grad(int nb, const int32_t* __restrict__ vertex, const double* __restrict__ target,
                               const double* __restrict__ compliance, const double* __restrict__ q,
                               const double* __restrict__ z, double h, double* d_target, double* d_compliance) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int v = vertex[b];
  const double e = compliance[b], k = h * h / e;
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double zr = z[3 * (size_t)v + r];
    if (d_target) d_target[3 * (size_t)b + r] = k * zr;
    s += zr * (q[3 * (size_t)v + r] - target[3 * (size_t)b + r]);
  }
  if (d_compliance) d_compliance[b] = k * s / e;
}

// ---- bindings of points inside tets: J_b q = sum_a w_a q_{tets[t][a]} (barycentric weights) ----
// (the blocks couple the vertices of one tet, so they land in the tet's own pattern slots)

// a tet id out of range, a weight that is not finite or a compliance that is not a positive finite
// number (FLAG_BADINDEX)
__global__ void k_check_bindings_bary(int nb, const int32_t* tet, const double* bary, const double* compliance,
                                      int nt, int* flags) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int t = tet[b];
  const double e = compliance[b];
  bool bad = t < 0 || t >= nt || !(e > 0.0) || !isfinite(e);
#pragma unroll
  for (int a = 0; a < 4; ++a) bad = bad || !isfinite(bary[4 * (size_t)b + a]);
  if (bad) atomicExch(&flags[FLAG_BADINDEX], 1);
}
// h^2 / E_b w_a w_c I_3 on the block (v_a, v_c) of the binding's tet
template <typename OutT>
__global__ void k_binding_blocks_bary(int nb, const int32_t* __restrict__ tet, const double* __restrict__ bary,
                                      const double* __restrict__ compliance, const int32_t* __restrict__ slot,
                                      double h, OutT* bsr) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int t = tet[b];
  const double k = h * h / compliance[b];
  double w[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) w[a] = bary[4 * (size_t)b + a];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double kac = k * w[a] * w[c];
      OutT* dst = bsr + 9 * (size_t)slot[16 * (size_t)t + 4 * a + c];
      atomic_add_out(dst + 0, kac);
      atomic_add_out(dst + 4, kac);
      atomic_add_out(dst + 8, kac);
    }
}
// the binding force: h^2 w_a (J_b q - d_b) / E_b at each vertex v_a of the tet
__global__ void k_binding_force_bary(int nb, const int32_t* __restrict__ tet, const int32_t* __restrict__ tets,
                                     const double* __restrict__ bary, const double* __restrict__ target,
                                     const double* __restrict__ compliance, const double* __restrict__ q, double h,
                                     double* R) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int t = tet[b];
  int v[4];
  double w[4], d[3] = {-target[3 * (size_t)b], -target[3 * (size_t)b + 1], -target[3 * (size_t)b + 2]};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    v[a] = tets[4 * (size_t)t + a];
    w[a] = bary[4 * (size_t)b + a];
#pragma unroll
    for (int r = 0; r < 3; ++r) d[r] += w[a] * q[3 * (size_t)v[a] + r];
  }
  const double k = h * h / compliance[b];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) atomicAdd(&R[3 * (size_t)v[a] + r], k * w[a] * d[r]);
}
// dL/dd_b = h^2 (J_b z) / E_b ; dL/dE_b = h^2 (J_b z) . (J_b q - d_b) / E_b^2
__global__ void k_binding_grad_bary(int nb, const int32_t* __restrict__ tet, const int32_t* __restrict__ tets,
                                    const double* __restrict__ bary, const double* __restrict__ target,
                                    const double* __restrict__ compliance, const double* __restrict__ q,
                                    const double* __restrict__ z, double h, double* d_target, double* d_compliance) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int t = tet[b];
  double jz[3] = {0.0, 0.0, 0.0}, d[3] = {-target[3 * (size_t)b], -target[3 * (size_t)b + 1], -target[3 * (size_t)b + 2]};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int v = tets[4 * (size_t)t + a];
    const double w = bary[4 * (size_t)b + a];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      jz[r] += w * z[3 * (size_t)v + r];
      d[r] += w * q[3 * (size_t)v + r];
    }
  }
  const double e = compliance[b], k = h * h / e;
  if (d_target) {
#pragma unroll
    for (int r = 0; r < 3; ++r) d_target[3 * (size_t)b + r] = k * jz[r];
  }
  if (d_compliance) d_compliance[b] = k * (jz[0] * d[0] + jz[1] * d[1] + jz[2] * d[2]) / e;
}

// ---- forward step ---------------------------------------------------------------------------

__global__ void k_predict(int nv, const double* q_prev, const double* v_prev, const double* f_ext, const double* mass,
                          double g0, double g1, double g2, double h, double* qt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nv) return;
  const int r = i % 3;
  double acc = (r == 0) ? g0 : (r == 1 ? g1 : g2);
  if (f_ext) acc += f_ext[i] / mass[i / 3];
  qt[i] = q_prev[i] + h * (v_prev ? v_prev[i] : 0.0) + h * h * acc;
}

__global__ void k_lift(int nc, const int32_t* vertex, const double* frame, const double* d_n, double gap0, double* q,
                       const double* q_prev, const double* d_f) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int v = vertex[c];
  const double* n = frame + 9 * (size_t)c;
  const double dn = n[0] * q[3 * v] + n[1] * q[3 * v + 1] + n[2] * q[3 * v + 2] - d_n[c];
  double d[3] = {0.0, 0.0, 0.0};
  if (dn < gap0)
    for (int r = 0; r < 3; ++r) d[r] = (gap0 - dn) * n[r];
  // a frictional contact needs a slip direction: where the prediction has exactly none (at rest
  // under a normal load), start from a 1e-12 m tangential offset in a direction fixed by c
  double s1 = 0.0, s2 = 0.0;
  for (int r = 0; r < 3; ++r) {
    const double dq = q[3 * v + r] - q_prev[3 * v + r];
    s1 += n[3 + r] * dq;
    s2 += n[6 + r] * dq;
  }
  if (d_f) {
    s1 -= d_f[2 * c];
    s2 -= d_f[2 * c + 1];
  }
  if (s1 == 0.0 && s2 == 0.0) {
    const double ang = 6.283185307179586 * (0.6180339887498949 * (double)(c + 1) - floor(0.6180339887498949 * (double)(c + 1)));
    const double a = 1e-12 * cos(ang), b = 1e-12 * sin(ang);
    for (int r = 0; r < 3; ++r) d[r] += a * n[3 + r] + b * n[6 + r];
  }
  for (int r = 0; r < 3; ++r)
    if (d[r] != 0.0) atomicAdd(&q[3 * v + r], d[r]);
}

__global__ void k_inertia(int nv, const double* mass, const double* q, const double* qt, double* R) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * nv) R[i] = mass[i / 3] * (q[i] - qt[i]);
}

__global__ void __launch_bounds__(128) k_tet_force(int nt, const int32_t* tets, const double* gvec,
                                                   const double* vol, const double* mu_, const double* lam_,
                                                   const int8_t* model, const double* q, double h, double* R,
                                                   int* flags) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int vid[4];
  double g[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    vid[a] = tets[4 * t + a];
#pragma unroll
    for (int k = 0; k < 3; ++k) g[a][k] = gvec[12 * t + 3 * a + k];
  }
  double F[3][3] = {};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) F[r][k] += q[3 * vid[a] + r] * g[a][k];
  double U[3][3], V[3][3], sig[3];
  if (!svd3<double>(F, U, sig, V)) {
    atomicExch(&flags[FLAG_INVERTED], 1);
    // also poison the tet's residual rows, so that a per-scene norm shows which scene it was
#pragma unroll
    for (int a = 0; a < 4; ++a) atomicAdd(&R[3 * (size_t)vid[a]], (double)INFINITY);
    return;
  }
  double th[3];
  local_theta<double>(model ? model[t] : MODEL_NEO_HOOKEAN, sig, mu_[t], lam_[t], th);
  // F - P = U diag(sigma - theta) V^T
  double D[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      D[r][k] = U[r][0] * (sig[0] - th[0]) * V[k][0] + U[r][1] * (sig[1] - th[1]) * V[k][1] +
                U[r][2] * (sig[2] - th[2]) * V[k][2];
  const double hw = h * h * 2.0 * mu_[t] * vol[t];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r)
      atomicAdd(&R[3 * vid[a] + r], hw * (D[r][0] * g[a][0] + D[r][1] * g[a][1] + D[r][2] * g[a][2]));
}

__global__ void k_local_contact(ContactArgs A, double* lambda, double* slip, int* loaded, double* R) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.nc) return;
  const int v = A.vertex[c];
  const double* F = A.frame + 9 * (size_t)c;
  double qv[3], dq[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    qv[r] = A.q[3 * v + r];
    dq[r] = qv[r] - A.q_prev[3 * v + r];
  }
  const double dn = F[0] * qv[0] + F[1] * qv[1] + F[2] * qv[2] - A.d_n[c];
  double df1 = F[3] * dq[0] + F[4] * dq[1] + F[5] * dq[2];
  double df2 = F[6] * dq[0] + F[7] * dq[1] + F[8] * dq[2];
  if (A.d_f) {
    df1 -= A.d_f[2 * c];
    df2 -= A.d_f[2 * c + 1];
  }
  const double e2 = A.eps * A.eps;
  const double mu = A.mu[c];
  const double s = sqrt(df1 * df1 + df2 * df2);
  slip[2 * c] = df1;
  slip[2 * c + 1] = df2;
  if (!(dn > 0.0) || (mu > 0.0 && !(s > 0.0))) {
    atomicExch(&A.flags[FLAG_INFEASIBLE], 1);
    if (loaded) loaded[c] = 0;
    if (R) atomicAdd(&R[3 * (size_t)v], (double)INFINITY);  // per-scene norms see it
    return;
  }
  const double lam_n = e2 / dn;
  double gam = 0.0, l1 = 0.0, l2 = 0.0;
  if (mu > 0.0) {
    gam = mu * lam_n - e2 / s;
    l1 = -gam * df1 / s;
    l2 = -gam * df2 / s;
  }
  if (loaded) loaded[c] = (mu > 0.0 && gam > 0.05 * mu * lam_n) ? 1 : 0;
  lambda[3 * c] = lam_n;
  lambda[3 * c + 1] = l1;
  lambda[3 * c + 2] = l2;
  const double h2 = A.h * A.h;
#pragma unroll
  for (int r = 0; r < 3; ++r) atomicAdd(&R[3 * v + r], -h2 * (F[r] * lam_n + F[3 + r] * l1 + F[6 + r] * l2));
}

__global__ void k_contact_scene(int nc, const int32_t* cv, const int32_t* sov, int32_t* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nc) out[c] = sov[cv[c]];
}
__global__ void k_scene_sq(int nv, const double* x, const int32_t* sov, double* sq) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double a = x[3 * v], b = x[3 * v + 1], c = x[3 * v + 2];
  atomicAdd(&sq[sov[v]], a * a + b * b + c * c);
}
__global__ void k_scale_by_scene(int nv, double* x, const int32_t* sov, const double* scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * nv) x[i] *= scale[sov[i / 3]];
}

__global__ void k_turn_check(int nc, const double* so, const double* sn, const int* loaded, int* flags,
                             const int32_t* cvertex, double* R) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc || !loaded[c]) return;
  const double d = so[2 * c] * sn[2 * c] + so[2 * c + 1] * sn[2 * c + 1];
  const double n0 = sqrt(so[2 * c] * so[2 * c] + so[2 * c + 1] * so[2 * c + 1]);
  const double n1 = sqrt(sn[2 * c] * sn[2 * c] + sn[2 * c + 1] * sn[2 * c + 1]);
  if (d < 0.5 * n0 * n1) {
    atomicExch(&flags[FLAG_TURN], 1);
    if (R) atomicAdd(&R[3 * (size_t)cvertex[c]], (double)INFINITY);
  }
}

// q_out[i] = q[i] + t[scene(vertex(i))] dx[i]
__global__ void k_step_by_scene(int nv, const double* q, const double* dx, const int32_t* sov, const double* t,
                                double* q_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * nv) q_out[i] = q[i] + t[sov[i / 3]] * dx[i];
}

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_check_contacts(int nc, const int32_t* vertex, const int32_t* region, int nv, int nreg, int* flags,
                           cudaStream_t s) {
  g_launches += 1;
  if (nc) k_check_contacts<<<nblk(nc, 128), 128, 0, s>>>(nc, vertex, region, nv, nreg, flags);
}

void launch_tet_assemble64(const TetArgs& a, cudaStream_t s) {
  g_launches += 1;
  if (a.nt) k_tet_assemble<double, double><<<nblk(a.nt, 128), 128, 0, s>>>(a, a.bsr);
}
void launch_tet_assemble32(const TetArgs& a, cudaStream_t s) {
  g_launches += 2;
  if (!a.nt) return;
  // FP32 Jacobian blocks; the contraction tensors (theta - sigma, dtheta/dmu, dtheta/dlambda, which lose
  // about three digits in FP32 at small strain) from an FP64 pass that skips the blocks
  TetArgs a32 = a;
  a32.tetdata = nullptr;
  k_tet_assemble<float, float><<<nblk(a.nt, 128), 128, 0, s>>>(a32, a.bsr32);
  k_tet_assemble<double, double><<<nblk(a.nt, 128), 128, 0, s>>>(a, (double*)nullptr);
}
void launch_contact_blocks(const ContactArgs& a, cudaStream_t s) {
  g_launches += 1;
  if (!a.nc) return;
  if (a.bsr) k_contact_blocks<double><<<nblk(a.nc, 128), 128, 0, s>>>(a, a.bsr);
  else k_contact_blocks<float><<<nblk(a.nc, 128), 128, 0, s>>>(a, a.bsr32);
}
void launch_bsr_init(int nv, int nb, const int32_t* diag_slot, const double* mass, double* bsr, float* bsr32,
                     cudaStream_t s) {
  g_launches += 2;
  if (bsr) {
    k_bsr_init<double><<<nblk(9L * nb, 256), 256, 0, s>>>(nv, nb, diag_slot, mass, bsr);
    k_bsr_mass<double><<<nblk(nv, 256), 256, 0, s>>>(nv, diag_slot, mass, bsr);
  }
  if (bsr32) {
    k_bsr_init<float><<<nblk(9L * nb, 256), 256, 0, s>>>(nv, nb, diag_slot, mass, bsr32);
    k_bsr_mass<float><<<nblk(nv, 256), 256, 0, s>>>(nv, diag_slot, mass, bsr32);
  }
}
// Actuation as a constant active stress P_i = a_i d_i d_i^T (fibre d_i, activation a_i): the nodal
// force f_a = -V_i P_i g_a = -V_i a_i (d_i . g_a) d_i is accumulated into f (which holds f_ext).
__global__ void k_act_force(int nt, const int32_t* __restrict__ tets, const double* __restrict__ gvec,
                            const double* __restrict__ vol, const float* __restrict__ act,
                            const double* __restrict__ fibre, double* f) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double s = -vol[t] * (double)act[t];
  if (s == 0.0) return;
  const double d0 = fibre[3 * (size_t)t], d1 = fibre[3 * (size_t)t + 1], d2 = fibre[3 * (size_t)t + 2];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double* g = gvec + 12 * (size_t)t + 3 * a;
    const double c = s * (d0 * g[0] + d1 * g[1] + d2 * g[2]);
    double* fv = f + 3 * (size_t)tets[4 * (size_t)t + a];
    atomicAdd(fv, c * d0);
    atomicAdd(fv + 1, c * d1);
    atomicAdd(fv + 2, c * d2);
  }
}

// dL/da_i = -h^2 V_i d_i^T Z_i d_i, Z_i = sum_a z_a g_a^T (the adjoint field's gradient on tet i)
__global__ void k_act_grad(int nt, const int32_t* __restrict__ tets, const double* __restrict__ gvec,
                           const double* __restrict__ vol, const double* __restrict__ fibre,
                           const double* __restrict__ z, double h, float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double d0 = fibre[3 * (size_t)t], d1 = fibre[3 * (size_t)t + 1], d2 = fibre[3 * (size_t)t + 2];
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double* g = gvec + 12 * (size_t)t + 3 * a;
    const double* za = z + 3 * (size_t)tets[4 * (size_t)t + a];
    acc += (d0 * za[0] + d1 * za[1] + d2 * za[2]) * (d0 * g[0] + d1 * g[1] + d2 * g[2]);
  }
  out[t] = (float)(-h * h * vol[t] * acc);
}

void launch_act_force(int nt, const int32_t* tets, const double* gvec, const double* vol, const float* act,
                      const double* fibre, double* f, cudaStream_t s) {
  g_launches += 1;
  if (nt) k_act_force<<<nblk(nt, 256), 256, 0, s>>>(nt, tets, gvec, vol, act, fibre, f);
}
void launch_act_grad(int nt, const int32_t* tets, const double* gvec, const double* vol, const double* fibre,
                     const double* z, double h, float* out, cudaStream_t s) {
  g_launches += 1;
  if (nt) k_act_grad<<<nblk(nt, 256), 256, 0, s>>>(nt, tets, gvec, vol, fibre, z, h, out);
}

void launch_predict(int nv, const double* q_prev, const double* v_prev, const double* f_ext, const double* mass,
                    double g0, double g1, double g2, double h, double* qt, cudaStream_t s) {
  g_launches += 1;
  k_predict<<<nblk(3L * nv, 256), 256, 0, s>>>(nv, q_prev, v_prev, f_ext, mass, g0, g1, g2, h, qt);
}
void launch_lift(int nc, const int32_t* vertex, const double* frame, const double* d_n, double gap0, double* q,
                 const double* q_prev, const double* d_f, cudaStream_t s) {
  g_launches += 1;
  if (nc) k_lift<<<nblk(nc, 128), 128, 0, s>>>(nc, vertex, frame, d_n, gap0, q, q_prev, d_f);
}
void launch_inertia(int nv, const double* mass, const double* q, const double* qt, double* R, cudaStream_t s) {
  g_launches += 1;
  k_inertia<<<nblk(3L * nv, 256), 256, 0, s>>>(nv, mass, q, qt, R);
}
void launch_check_bindings(int nb, const int32_t* vertex, const double* compliance, int nv, int* flags,
                           cudaStream_t s) {
  g_launches += 1;
  if (nb) k_check_bindings<<<nblk(nb, 128), 128, 0, s>>>(nb, vertex, compliance, nv, flags);
}
void launch_binding_blocks(int nb, const int32_t* vertex, const double* compliance, const int32_t* diag_slot,
                           double h, double* bsr, float* bsr32, cudaStream_t s) {
  g_launches += 1;
  if (!nb) return;
  if (bsr) k_binding_blocks<double><<<nblk(nb, 128), 128, 0, s>>>(nb, vertex, compliance, diag_slot, h, bsr);
  else k_binding_blocks<float><<<nblk(nb, 128), 128, 0, s>>>(nb, vertex, compliance, diag_slot, h, bsr32);
}
void launch_binding_force(int nb, const int32_t* vertex, const double* target, const double* compliance,
                          const double* q, double h, double* R, cudaStream_t s) {
  g_launches += 1;
  if (nb) k_binding_force<<<nblk(nb, 128), 128, 0, s>>>(nb, vertex, target, compliance, q, h, R);
}
void launch_binding_grad(int nb, const int32_t* vertex, const double* target, const double* compliance,
                         const double* q, const double* z, double h, double* d_target, double* d_compliance,
                         cudaStream_t s) {
  g_launches += 1;
  if (nb) k_binding_grad<<<nblk(nb, 128), 128, 0, s>>>(nb, vertex, target, compliance, q, z, h, d_target, d_compliance);
}
void launch_check_bindings_bary(int nb, const int32_t* tet, const double* bary, const double* compliance, int nt,
                                int* flags, cudaStream_t s) {
  g_launches += 1;
  if (nb) k_check_bindings_bary<<<nblk(nb, 128), 128, 0, s>>>(nb, tet, bary, compliance, nt, flags);
}
void launch_binding_blocks_bary(int nb, const int32_t* tet, const double* bary, const double* compliance,
                                const int32_t* slot, double h, double* bsr, float* bsr32, cudaStream_t s) {
  g_launches += 1;
  if (!nb) return;
  if (bsr) k_binding_blocks_bary<double><<<nblk(nb, 128), 128, 0, s>>>(nb, tet, bary, compliance, slot, h, bsr);
  else k_binding_blocks_bary<float><<<nblk(nb, 128), 128, 0, s>>>(nb, tet, bary, compliance, slot, h, bsr32);
}
void launch_binding_force_bary(int nb, const int32_t* tet, const int32_t* tets, const double* bary,
                               const double* target, const double* compliance, const double* q, double h, double* R,
                               cudaStream_t s) {
  g_launches += 1;
  if (nb) k_binding_force_bary<<<nblk(nb, 128), 128, 0, s>>>(nb, tet, tets, bary, target, compliance, q, h, R);
}
void launch_binding_grad_bary(int nb, const int32_t* tet, const int32_t* tets, const double* bary,
                              const double* target, const double* compliance, const double* q, const double* z,
                              double h, double* d_target, double* d_compliance, cudaStream_t s) {
  g_launches += 1;
  if (nb)
    k_binding_grad_bary<<<nblk(nb, 128), 128, 0, s>>>(nb, tet, tets, bary, target, compliance, q, z, h, d_target,
                                                       d_compliance);
}
void launch_tet_force(int nt, const int32_t* tets, const double* gvec, const double* vol, const double* mu,
                      const double* lam, const int8_t* model, const double* q, double h, double* R, int* flags,
                      cudaStream_t s) {
  g_launches += 1;
  if (nt) k_tet_force<<<nblk(nt, 128), 128, 0, s>>>(nt, tets, gvec, vol, mu, lam, model, q, h, R, flags);
}
void launch_local_contact(const ContactArgs& a, double* lambda, double* slip, int* loaded, double* R,
                          cudaStream_t s) {
  g_launches += 1;
  if (a.nc) k_local_contact<<<nblk(a.nc, 128), 128, 0, s>>>(a, lambda, slip, loaded, R);
}
void launch_contact_scene(int nc, const int32_t* cvertex, const int32_t* sov, int32_t* out, cudaStream_t s) {
  g_launches += 1;
  if (nc) k_contact_scene<<<nblk(nc, 128), 128, 0, s>>>(nc, cvertex, sov, out);
}
void launch_scene_sq(int nv, const double* x, const int32_t* sov, double* sq, cudaStream_t s) {
  g_launches += 1;
  k_scene_sq<<<nblk(nv, 256), 256, 0, s>>>(nv, x, sov, sq);
}
void launch_scale_by_scene(int nv, double* x, const int32_t* sov, const double* scale, cudaStream_t s) {
  g_launches += 1;
  k_scale_by_scene<<<nblk(3L * nv, 256), 256, 0, s>>>(nv, x, sov, scale);
}
void launch_step_by_scene(int nv, const double* q, const double* dx, const int32_t* sov, const double* t,
                          double* q_out, cudaStream_t s) {
  g_launches += 1;
  k_step_by_scene<<<nblk(3L * nv, 256), 256, 0, s>>>(nv, q, dx, sov, t, q_out);
}
void launch_turn_check(int nc, const double* slip_old, const double* slip_new, const int* loaded, int* flags,
                       const int32_t* cvertex, double* R, cudaStream_t s) {
  g_launches += 1;
  if (nc) k_turn_check<<<nblk(nc, 128), 128, 0, s>>>(nc, slip_old, slip_new, loaded, flags, cvertex, R);
}
void launch_contractions(const ContractArgs& a, cudaStream_t s) {
  g_launches += 3;
  k_contract_vertex<<<nblk(3L * a.nv, 256), 256, 0, s>>>(a);
  if (a.nc) k_contract_contact<<<nblk(a.nc, 128), 128, 0, s>>>(a);
  if (a.nt) k_contract_tet<<<nblk(a.nt, 128), 128, 0, s>>>(a);
}

}  // namespace ncpadj
