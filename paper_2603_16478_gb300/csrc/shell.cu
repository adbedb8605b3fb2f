// Triangle (shell) elements and isometric bending: the 2D formulation of App. B.1.
//
//  * tri_assemble: F = D_s D_m^{-1} (3 x 2, D_m the rest edges in the triangle's own plane), its
//    thin SVD F = U diag(sigma) V^T (U 3 x 2 completed by the unit normal u_3 = u_1 x u_2, V 2 x 2),
//    theta(sigma) of the element's model with W = dtheta/dsigma, and the projection Jacobian
//    dvecP/dvecF in the SVD closed form of the tets (diagonal W, in-plane pair through the
//    coefficients M, N of App. B.0) plus the out-of-plane rows: a perturbation of F along the normal,
//    X_3j, moves P along the normal by (theta_j / sigma_j) X_3j.  The Jacobian is folded into the 6
//    unique 3x3 blocks of h^2 w_i G_i^T (I - dP/dF) G_i, w_i = 2 mu_i A_i tau (tau: thickness).
//  * tri_force: the elastic part of the forward residual, h^2 w_i G_i^T vec(F - P).
//  * contract_tri: dL/dE, dL/dnu of each triangle (App. B.3 with the 3 x 2 tensors).
//  * bend_*: isometric bending (Bergou, Wardetzky, Harmon, Zorin, Grinspun 2006): per interior
//    edge e with the cotangent stencil K of its 4 vertices, the energy 1/2 k_b (3/(A_1+A_2)) |sum_a
//    K_a x_a|^2; a constant Hessian h^2 k_b Q_e (x) I_3 in script_A, the force h^2 k_b Q q in the
//    forward residual and dL/dk_b = -h^2 z^T Q q per mesh.
#include <math.h>

#include "kernels.cuh"

namespace ncpadj {
namespace {

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

template <typename T> struct Sh;
template <> struct Sh<double> {
  static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
  static __device__ __forceinline__ double lg(double x) { return log(x); }
  static constexpr double tol_newton = 1e-14;
};
template <> struct Sh<float> {
  static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float lg(float x) { return logf(x); }
  static constexpr float tol_newton = 2e-6f;
};

// Thin SVD of a 3 x 2 F through the symmetric Schur decomposition of C = F^T F (one exact Jacobi
// rotation, Golub & Van Loan Sec. 8.5): V its eigenvectors, sigma = sqrt(eigenvalues),
// u_j = F v_j / sigma_j, u_3 = u_1 x u_2.  False when F has rank < 2 (or is not finite).
template <typename T>
__device__ bool svd32(const T F[3][2], T U[3][3], T sig[2], T V[2][2]) {
  const T a = F[0][0] * F[0][0] + F[1][0] * F[1][0] + F[2][0] * F[2][0];
  const T b = F[0][0] * F[0][1] + F[1][0] * F[1][1] + F[2][0] * F[2][1];
  const T c = F[0][1] * F[0][1] + F[1][1] * F[1][1] + F[2][1] * F[2][1];
  T cs = T(1), sn = T(0), e0 = a, e1 = c;
  if (b != T(0)) {
    const T tau = (c - a) / (T(2) * b);
    const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + Sh<T>::sq(T(1) + tau * tau));
    cs = T(1) / Sh<T>::sq(T(1) + t * t);
    sn = t * cs;
    e0 = a - t * b;
    e1 = c + t * b;
  }
  if (!(e0 > T(0) && e1 > T(0)) || !isfinite(e0 + e1)) return false;
  sig[0] = Sh<T>::sq(e0);
  sig[1] = Sh<T>::sq(e1);
  V[0][0] = cs;
  V[1][0] = -sn;
  V[0][1] = sn;
  V[1][1] = cs;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int r = 0; r < 3; ++r) U[r][j] = (F[r][0] * V[0][j] + F[r][1] * V[1][j]) / sig[j];
  U[0][2] = U[1][0] * U[2][1] - U[2][0] * U[1][1];
  U[1][2] = U[2][0] * U[0][1] - U[0][0] * U[2][1];
  U[2][2] = U[0][0] * U[1][1] - U[1][0] * U[0][1];
  const T nn = Sh<T>::sq(U[0][2] * U[0][2] + U[1][2] * U[1][2] + U[2][2] * U[2][2]);
#pragma unroll
  for (int r = 0; r < 3; ++r) U[r][2] /= nn;
  return true;
}

// The 2D singular-value projection of the three models, with W = dtheta/dsigma, the total
// dtheta/dmu and dtheta/dlambda (w = 2 mu varies with mu) and the divided difference
// Ad = (theta_0 - theta_1)/(sigma_0 - sigma_1) in a form without cancellation.  The stationarity
// conditions are those of the volumetric models with two singular values:
//  - Neo-Hookean: mu (3 theta_i - 2 sigma_i - 1/theta_i) + lambda log(J) / theta_i = 0, J = theta_0
//    theta_1, by damped Newton from theta = sigma (Hessian diag + lambda a a^T, a = 1/theta, inverted
//    by Sherman-Morrison); Ad = 2 mu / (3 mu + (mu - lambda log J) / (theta_0 theta_1));
//  - co-rotational: theta = (sigma + 1)/2 - c sum(sigma - 1), c = lambda / (2 (4 mu + 2 lambda));
//    W = I/2 - c 1 1^T, Ad = 1/2;
//  - ARAP: theta = 1, W = 0, Ad = 0.
template <typename T>
__device__ void local_prox2(int model, const T sig[2], T mu, T lam, T th[2], T W[2][2], T dmu[2], T dlam[2],
                            T& Ad) {
  if (model == MODEL_COROTATIONAL) {
    const T den = T(4) * mu + T(2) * lam;
    const T c = lam / (T(2) * den);
    const T s = (sig[0] - T(1)) + (sig[1] - T(1));
    const T gm = T(2) * lam * s / (den * den), gl = -T(2) * mu * s / (den * den);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      th[i] = T(0.5) * (sig[i] + T(1)) - c * s;
      dmu[i] = gm;
      dlam[i] = gl;
#pragma unroll
      for (int j = 0; j < 2; ++j) W[i][j] = (i == j ? T(0.5) : T(0)) - c;
    }
    Ad = T(0.5);
    return;
  }
  if (model == MODEL_ARAP) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      th[i] = T(1);
      dmu[i] = dlam[i] = T(0);
      W[i][0] = W[i][1] = T(0);
    }
    Ad = T(0);
    return;
  }
  th[0] = sig[0];
  th[1] = sig[1];
  T logJ = T(0), a[2], Dg[2];
  for (int it = 0; it < 40; ++it) {
    logJ = Sh<T>::lg(th[0] * th[1]);
    T g[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      a[i] = T(1) / th[i];
      g[i] = mu * (T(3) * th[i] - T(2) * sig[i] - a[i]) + lam * logJ * a[i];
    }
    if (fmax(fabs(g[0]), fabs(g[1])) <= Sh<T>::tol_newton * mu) break;
    T Dia[2], Dig[2], aDa = 0, aDg = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      Dg[i] = T(3) * mu + (mu - lam * logJ) * a[i] * a[i];
      Dia[i] = a[i] / Dg[i];
      Dig[i] = g[i] / Dg[i];
      aDa += a[i] * Dia[i];
      aDg += a[i] * Dig[i];
    }
    const T coef = lam * aDg / (T(1) + lam * aDa);
    T step[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) step[i] = -(Dig[i] - coef * Dia[i]);
    T t = T(1);
    for (int k = 0; k < 30; ++k) {
      if (th[0] + t * step[0] > T(0) && th[1] + t * step[1] > T(0)) break;
      t *= T(0.5);
    }
    th[0] += t * step[0];
    th[1] += t * step[1];
  }
  logJ = Sh<T>::lg(th[0] * th[1]);
  T Dia[2], aDa = 0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    a[i] = T(1) / th[i];
    Dg[i] = T(3) * mu + (mu - lam * logJ) * a[i] * a[i];
    Dia[i] = a[i] / Dg[i];
    aDa += a[i] * Dia[i];
  }
  const T cc = lam / (T(1) + lam * aDa);
  T Hinv[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) Hinv[i][j] = ((i == j) ? T(1) / Dg[i] : T(0)) - cc * Dia[i] * Dia[j];
  T gm[2], gl[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    gm[i] = T(3) * th[i] - T(2) * sig[i] - T(1) / th[i];
    gl[i] = logJ / th[i];
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    dmu[i] = -(Hinv[i][0] * gm[0] + Hinv[i][1] * gm[1]);
    dlam[i] = -(Hinv[i][0] * gl[0] + Hinv[i][1] * gl[1]);
    W[i][0] = T(2) * mu * Hinv[i][0];
    W[i][1] = T(2) * mu * Hinv[i][1];
  }
  Ad = T(2) * mu / (T(3) * mu + (mu - lam * logJ) / (th[0] * th[1]));
}

template <typename T>
__device__ __forceinline__ void add_out(double* p, T v) { atomicAdd(p, (double)v); }
template <typename T>
__device__ __forceinline__ void add_out(float* p, T v) { atomicAdd(p, (float)v); }

// F = sum_a x_a g_a^T of triangle t (g_a: 2-vectors, gvec [nt][6])
template <typename T>
__device__ __forceinline__ void tri_F(const int32_t* tris, const double* gvec, const double* q, int t, int vid[3],
                                      T g[3][2], T F[3][2]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vid[a] = tris[3 * t + a];
    g[a][0] = (T)gvec[6 * t + 2 * a];
    g[a][1] = (T)gvec[6 * t + 2 * a + 1];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) F[r][0] = F[r][1] = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T x = (T)q[3 * vid[a] + r];
      F[r][0] += x * g[a][0];
      F[r][1] += x * g[a][1];
    }
}

// TetArgs with the triangle layout: tets [nt][3], gvec [nt][6], slot [nt][9], tetdata [nt][12]
template <typename T, typename OutT>
__global__ void __launch_bounds__(128) k_tri_assemble(TetArgs A, OutT* bsr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.nt) return;
  int vid[3];
  T g[3][2], F[3][2];
  tri_F<T>(A.tets, A.gvec, A.q, t, vid, g, F);
  T U[3][3], V[2][2], sig[2];
  if (!svd32<T>(F, U, sig, V)) {
    atomicExch(&A.flags[FLAG_INVERTED], 1);
    return;
  }
  const T mu = (T)A.mu[t], lam = (T)A.lam[t];
  T th[2], W[2][2], dmu[2], dlam[2], Ad;
  local_prox2<T>(A.model ? A.model[t] : MODEL_NEO_HOOKEAN, sig, mu, lam, th, W, dmu, dlam, Ad);
  if (bsr != nullptr) {
    const T Bd = (th[0] + th[1]) / (sig[0] + sig[1]);
    const T Mc = T(0.5) * (Ad + Bd), Nc = T(0.5) * (Ad - Bd);
    const T r0 = th[0] / sig[0], r1 = th[1] / sig[1];
    T c[2][3];  // c_j[a] = g_a . v_j
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int a = 0; a < 3; ++a) c[j][a] = g[a][0] * V[0][j] + g[a][1] * V[1][j];
    const T hw = (T)(A.h * A.h) * T(2) * mu * (T)A.vol[t];
    // block (a, b) = hw U Q U^T with, in the basis (u_1, u_2, n):
    //   Q_pp = g_a.g_b - W_pp c_p[a] c_p[b] - M c_o[a] c_o[b]        (p in-plane, o the other)
    //   Q_po = -W_po c_p[a] c_o[b] - N c_o[a] c_p[b]
    //   Q_nn = g_a.g_b - sum_j (theta_j / sigma_j) c_j[a] c_j[b],  Q_pn = Q_np = 0
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
#pragma unroll 1
      for (int b = a; b < 3; ++b) {
        const T p0 = c[0][a] * c[0][b], p1 = c[1][a] * c[1][b];
        const T gg = p0 + p1;
        T Q[3][3] = {};
        Q[0][0] = gg - W[0][0] * p0 - Mc * p1;
        Q[1][1] = gg - W[1][1] * p1 - Mc * p0;
        Q[0][1] = -W[0][1] * c[0][a] * c[1][b] - Nc * c[1][a] * c[0][b];
        Q[1][0] = -W[1][0] * c[1][a] * c[0][b] - Nc * c[0][a] * c[1][b];
        Q[2][2] = gg - r0 * p0 - r1 * p1;
        T UQ[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int k = 0; k < 3; ++k) UQ[r][k] = U[r][0] * Q[0][k] + U[r][1] * Q[1][k] + U[r][2] * Q[2][k];
        T blk[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int s = 0; s < 3; ++s) blk[r][s] = hw * (UQ[r][0] * U[s][0] + UQ[r][1] * U[s][1] + UQ[r][2] * U[s][2]);
        OutT* dst = bsr + 9 * (size_t)A.slot[9 * t + 3 * a + b];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int s = 0; s < 3; ++s) add_out(dst + 3 * r + s, blk[r][s]);
        if (a != b) {
          OutT* dst2 = bsr + 9 * (size_t)A.slot[9 * t + 3 * b + a];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = 0; s < 3; ++s) add_out(dst2 + 3 * r + s, blk[s][r]);
        }
      }
    }
  }
  if (A.tetdata == nullptr) return;
  // contraction tensors P_mu = U diag(e_mu) V^T, P_lam = U diag(e_lam) V^T (3 x 2, row-major) with
  // e_mu = 2 h^2 A tau (mu dtheta/dmu + theta - sigma), e_lam = 2 h^2 A tau mu dtheta/dlambda
  const double h2v2 = 2.0 * A.h * A.h * A.vol[t];
  double em[2], el[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    em[i] = h2v2 * ((double)mu * dmu[i] + (double)th[i] - (double)sig[i]);
    el[i] = h2v2 * (double)mu * dlam[i];
  }
  double* td = A.tetdata + 12 * (size_t)t;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double u0 = (double)U[r][0] * (double)V[k][0], u1 = (double)U[r][1] * (double)V[k][1];
      td[2 * r + k] = em[0] * u0 + em[1] * u1;
      td[6 + 2 * r + k] = el[0] * u0 + el[1] * u1;
    }
}

__global__ void __launch_bounds__(128) k_tri_force(int nt, const int32_t* tris, const double* gvec, const double* vol,
                                                   const double* mu_, const double* lam_, const int8_t* model,
                                                   const double* q, double h, double* R, int* flags) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int vid[3];
  double g[3][2], F[3][2];
  tri_F<double>(tris, gvec, q, t, vid, g, F);
  double U[3][3], V[2][2], sig[2];
  if (!svd32<double>(F, U, sig, V)) {
    atomicExch(&flags[FLAG_INVERTED], 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) atomicAdd(&R[3 * (size_t)vid[a]], (double)INFINITY);
    return;
  }
  double th[2], W[2][2], dmu[2], dlam[2], Ad;
  local_prox2<double>(model ? model[t] : MODEL_NEO_HOOKEAN, sig, mu_[t], lam_[t], th, W, dmu, dlam, Ad);
  double D[3][2];  // F - P = U diag(sigma - theta) V^T
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 2; ++k) D[r][k] = U[r][0] * (sig[0] - th[0]) * V[k][0] + U[r][1] * (sig[1] - th[1]) * V[k][1];
  const double hw = h * h * 2.0 * mu_[t] * vol[t];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) atomicAdd(&R[3 * vid[a] + r], hw * (D[r][0] * g[a][0] + D[r][1] * g[a][1]));
}

__global__ void k_contract_tri(ContractArgs A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.nt) return;
  const double* td = A.tetdata + 12 * (size_t)t;
  const double* g = A.gvec + 6 * (size_t)t;
  double dmu = 0, dlam = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int v = A.tets[3 * t + a];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double za = A.z[3 * v + r];
      dmu += za * (td[2 * r] * g[2 * a] + td[2 * r + 1] * g[2 * a + 1]);
      dlam += za * (td[6 + 2 * r] * g[2 * a] + td[6 + 2 * r + 1] * g[2 * a + 1]);
    }
  }
  const double* ld = A.lame_d + 4 * (size_t)t;
  if (A.dL_dE) A.dL_dE[t] = dmu * ld[0] + dlam * ld[1];
  if (A.dL_dnu) A.dL_dnu[t] = dmu * ld[2] + dlam * ld[3];
}

// ---- isometric bending ------------------------------------------------------------------------
// hinge e: vertices idx[4e..4e+3], coefficients coef[5e..5e+4] = (K_0..K_3, 3/(A_1+A_2)), the
// stiffness kb[e] of its mesh, block slots slot[16e + 4a + b]
template <typename OutT>
__global__ void k_bend_blocks(int ne, const int32_t* __restrict__ idx, const double* __restrict__ coef,
                              const double* __restrict__ kb, const int32_t* __restrict__ slot, double h, OutT* bsr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double* k = coef + 5 * (size_t)e;
  const double s = h * h * kb[e] * k[4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      OutT* dst = bsr + 9 * (size_t)slot[16 * e + 4 * a + b];
      const OutT v = (OutT)(s * k[a] * k[b]);
      atomicAdd(dst, v);
      atomicAdd(dst + 4, v);
      atomicAdd(dst + 8, v);
    }
}

__global__ void k_bend_force(int ne, const int32_t* __restrict__ idx, const double* __restrict__ coef,
                             const double* __restrict__ kb, const double* __restrict__ q, double h, double* R) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double* k = coef + 5 * (size_t)e;
  const int32_t* v = idx + 4 * (size_t)e;
  double y[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) y[r] += k[a] * q[3 * v[a] + r];
  const double s = h * h * kb[e] * k[4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) atomicAdd(&R[3 * v[a] + r], s * k[a] * y[r]);
}

// dL/dk_b of mesh blockIdx.x = -h^2 sum_e (3/(A_1+A_2)) (K z) . (K q) over its hinges
// [eoff[s], eoff[s+1]) (one block per mesh: a fixed summation order)
__global__ void __launch_bounds__(256) k_bend_grad(const int32_t* __restrict__ eoff, const int32_t* __restrict__ idx,
                                                   const double* __restrict__ coef, const double* __restrict__ q,
                                                   const double* __restrict__ z, double h, double* out) {
  __shared__ double red[256];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int e = eoff[s] + threadIdx.x; e < eoff[s + 1]; e += blockDim.x) {
    const double* k = coef + 5 * (size_t)e;
    const int32_t* v = idx + 4 * (size_t)e;
    double yq[3] = {0, 0, 0}, yz[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        yq[r] += k[a] * q[3 * v[a] + r];
        yz[r] += k[a] * z[3 * v[a] + r];
      }
    acc += k[4] * (yq[0] * yz[0] + yq[1] * yz[1] + yq[2] * yz[2]);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[s] = -h * h * red[0];
}

}  // namespace

void launch_tri_assemble64(const TetArgs& a, cudaStream_t s) {
  g_launches += 1;
  if (a.nt) k_tri_assemble<double, double><<<nblk(a.nt, 128), 128, 0, s>>>(a, a.bsr);
}
void launch_tri_assemble32(const TetArgs& a, cudaStream_t s) {
  g_launches += 2;
  if (!a.nt) return;
  // FP32 blocks; the contraction tensors from an FP64 pass that skips the blocks (as for tets)
  TetArgs b = a;
  b.tetdata = nullptr;
  k_tri_assemble<float, float><<<nblk(a.nt, 128), 128, 0, s>>>(b, a.bsr32);
  if (a.tetdata) k_tri_assemble<double, double><<<nblk(a.nt, 128), 128, 0, s>>>(a, static_cast<double*>(nullptr));
}
void launch_tri_force(int nt, const int32_t* tris, const double* gvec, const double* vol, const double* mu,
                      const double* lam, const int8_t* model, const double* q, double h, double* R, int* flags,
                      cudaStream_t s) {
  g_launches += 1;
  if (nt) k_tri_force<<<nblk(nt, 128), 128, 0, s>>>(nt, tris, gvec, vol, mu, lam, model, q, h, R, flags);
}
void launch_contract_tri(const ContractArgs& a, cudaStream_t s) {
  g_launches += 1;
  if (a.nt) k_contract_tri<<<nblk(a.nt, 128), 128, 0, s>>>(a);
}
void launch_bend_blocks(int ne, const int32_t* idx, const double* coef, const double* kb, const int32_t* slot,
                        double h, double* bsr, float* bsr32, cudaStream_t s) {
  if (!ne) return;
  g_launches += 1;
  if (bsr32) k_bend_blocks<float><<<nblk(ne, 128), 128, 0, s>>>(ne, idx, coef, kb, slot, h, bsr32);
  else k_bend_blocks<double><<<nblk(ne, 128), 128, 0, s>>>(ne, idx, coef, kb, slot, h, bsr);
}
void launch_bend_force(int ne, const int32_t* idx, const double* coef, const double* kb, const double* q, double h,
                       double* R, cudaStream_t s) {
  if (!ne) return;
  g_launches += 1;
  k_bend_force<<<nblk(ne, 128), 128, 0, s>>>(ne, idx, coef, kb, q, h, R);
}
void launch_bend_grad(int n_scenes, const int32_t* eoff, const int32_t* idx, const double* coef, const double* q,
                      const double* z, double h, double* out, cudaStream_t s) {
  g_launches += 1;
  k_bend_grad<<<n_scenes, 256, 0, s>>>(eoff, idx, coef, q, z, h, out);
}

}  // namespace ncpadj
