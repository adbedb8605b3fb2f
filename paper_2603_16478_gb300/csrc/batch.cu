// Vector kernels of the batched adjoint: one restarted GMRES per scene of a batch (Sec. 4.4, the
// Krylov solve of Eq. adjoint), all scenes advanced by the same launches.
//
// A batch scene is the disjoint union of independent meshes, so its adjoint matrix, its
// preconditioner and their products are block-diagonal by scene.  What couples the scenes in a
// single Krylov solve over the union is only the inner products; here every inner product, norm,
// Hessenberg column, Givens rotation and stopping test is per scene.  The union's DOF range is cut
// into tiles that never straddle two scenes; a reduction over a scene sums its tiles' partials in
// tile order (deterministic), done by the last of its blocks to finish.  A scene leaves the step's
// work (act[s] = 0) as soon as its own residual estimate meets its own tolerance: every kernel of
// a step, the preconditioner and the matrix product included, skips its rows.
#include <math.h>

#include "dfloat.cuh"
#include "kernels.cuh"

namespace ncpadj {

namespace {

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of a value over the 256 threads of a block, in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ double block_sum256(double v, double* sh) {
  v = wsum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < 8; ++i) r += sh[i];
  return r;
}

// Tile t's partial of reduction k goes to partial[k][t]; the last tile of scene s to arrive (counter
// cnt[s][slot], which it resets) adds the scene's partials in tile order and writes *out.
__device__ void seg_finish(double acc, const SegTiles& T, int t, int s, int k, unsigned* cnt, int slot, int K,
                           double* partial, double* out) {
  __shared__ double sh[8];
  __shared__ bool last;
  const double v = block_sum256(acc, sh);
  if (threadIdx.x == 0) {
    partial[(size_t)k * T.n + t] = v;
    __threadfence();
    const unsigned ntile = (unsigned)(T.t0[s + 1] - T.t0[s]);
    last = atomicAdd(&cnt[(size_t)s * K + slot], 1u) == ntile - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double u = 0.0;
  for (int i = T.t0[s] + (int)threadIdx.x; i < T.t0[s + 1]; i += blockDim.x) u += __ldcg(&partial[(size_t)k * T.n + i]);
  __syncthreads();  // sh is reused
  const double r = block_sum256(u, sh);
  if (threadIdx.x == 0) {
    *out = r;
    cnt[(size_t)s * K + slot] = 0;
  }
}

// Step j = *jp of the scenes' Arnoldi processes: gsb[s][goff + k] = V_k . V_{j+1} over scene s's
// DOFs for k <= j (blockIdx.y = k), or with self gsb[s][goff] = |V_{j+1}|^2.
__global__ void __launch_bounds__(256) k_seg_dot_step(SegTiles T, const double* __restrict__ V, long ld,
                                                      const int* __restrict__ jp, int m, int self,
                                                      const int* __restrict__ act, double* partial, unsigned* cnt,
                                                      int K, double* gsb, int gstride, int goff) {
  const int j = *jp;
  if (j >= m) return;
  const int t = blockIdx.x, k = blockIdx.y, s = T.scene[t];
  if (k > (self ? 0 : j) || !act[s]) return;
  const double* w = V + (size_t)(j + 1) * ld;
  const double* a = self ? w : V + (size_t)k * ld;
  double acc = 0.0;
  for (int i = T.beg[t] + (int)threadIdx.x; i < T.end[t]; i += blockDim.x) acc += a[i] * w[i];
  seg_finish(acc, T, t, s, k, cnt, self ? m + 1 : k, K, partial, gsb + (size_t)s * gstride + goff + k);
}

// out[s] = |x|^2 over scene s's DOFs, for the scenes with mask[s]
__global__ void __launch_bounds__(256) k_seg_sq(SegTiles T, const double* __restrict__ x,
                                                const int* __restrict__ mask, double* partial, unsigned* cnt, int K,
                                                int slot, double* out) {
  const int t = blockIdx.x, s = T.scene[t];
  if (!mask[s]) return;
  double acc = 0.0;
  for (int i = T.beg[t] + (int)threadIdx.x; i < T.end[t]; i += blockDim.x) acc += x[i] * x[i];
  seg_finish(acc, T, t, s, 0, cnt, slot, K, partial, out + s);
}

// V_{j+1} -= sum_{k <= j} gsb[s][goff + k] V_k on scene s's tiles
__global__ void __launch_bounds__(256) k_seg_axpy_step(SegTiles T, double* __restrict__ V, long ld,
                                                       const int* __restrict__ jp, int m,
                                                       const int* __restrict__ act, const double* __restrict__ gsb,
                                                       int gstride, int goff) {
  const int j = *jp;
  if (j >= m) return;
  const int t = blockIdx.x, s = T.scene[t];
  if (!act[s]) return;
  __shared__ double c[kMaxRestart + 1];
  for (int k = threadIdx.x; k <= j; k += blockDim.x) c[k] = gsb[(size_t)s * gstride + goff + k];
  __syncthreads();
  double* w = V + (size_t)(j + 1) * ld;
  for (int i = T.beg[t] + (int)threadIdx.x; i < T.end[t]; i += blockDim.x) {
    double acc = w[i];
    for (int k = 0; k <= j; ++k) acc -= c[k] * V[(size_t)k * ld + i];
    w[i] = acc;
  }
}

// V_{j+1} /= sqrt(gsb[s][noff]) (a zero or non-finite norm leaves a zero vector)
__global__ void __launch_bounds__(256) k_seg_normalize_step(SegTiles T, double* __restrict__ V, long ld,
                                                            const int* __restrict__ jp, int m,
                                                            const int* __restrict__ act,
                                                            const double* __restrict__ gsb, int gstride, int noff) {
  const int j = *jp;
  if (j >= m) return;
  const int t = blockIdx.x, s = T.scene[t];
  if (!act[s]) return;
  const double nr = sqrt(gsb[(size_t)s * gstride + noff]);
  const double inv = (nr > 0.0 && isfinite(nr)) ? 1.0 / nr : 0.0;
  double* w = V + (size_t)(j + 1) * ld;
  for (int i = T.beg[t] + (int)threadIdx.x; i < T.end[t]; i += blockDim.x) w[i] = inv > 0.0 ? w[i] * inv : 0.0;
}

// dst = src, or dst = d .* src when d is given, on the tiles of active scenes; src is taken at
// src + j ld when src_idx, dst at dst + j ld when dst_idx (j = *jp); with split, also the
// double-float pairs of dst (the input of the double-float block product)
__global__ void __launch_bounds__(256) k_seg_copy_step(SegTiles T, const double* __restrict__ src, int src_idx,
                                                       double* __restrict__ dst, int dst_idx, long ld,
                                                       const int* __restrict__ jp, int m, const int* __restrict__ act,
                                                       const double* __restrict__ d, float2* __restrict__ split) {
  const int j = *jp;
  if (j >= m) return;
  const int t = blockIdx.x, s = T.scene[t];
  if (!act[s]) return;
  if (src_idx) src += (size_t)j * ld;
  if (dst_idx) dst += (size_t)j * ld;
  for (int i = T.beg[t] + (int)threadIdx.x; i < T.end[t]; i += blockDim.x) {
    const double v = d ? d[i] * src[i] : src[i];
    dst[i] = v;
    if (split) split[i] = df_split(v);
  }
}

// The Hessenberg column of step j of every active scene (first- plus second-pass Gram-Schmidt
// coefficients, the new vector's norm), its Givens rotations and residual estimate |g_{j+1}|.  A
// scene stops for the rest of the cycle when the estimate is at most tol[s], when it reaches
// maxit iterations, or at the end of the cycle (j + 1 = m).  One block; then the number of scenes
// still active goes to the host-mapped nact[j] and *jp = j + 1.
__global__ void __launch_bounds__(256) k_seg_givens(int ns, int* jp, int m, int* act, const double* __restrict__ gsb,
                                                    int gstride, double* H, double* cs, double* sn, double* g, int* kk,
                                                    int* iters, const double* __restrict__ tol, int maxit,
                                                    volatile int* nact) {
  const int j = *jp;
  if (j >= m) return;
  __shared__ double sh[8];
  double live = 0.0;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    if (!act[s]) continue;
    const double* gg = gsb + (size_t)s * gstride;
    double* hc = H + (size_t)s * (m + 1) * m + (size_t)(m + 1) * j;
    double* c = cs + (size_t)s * m;
    double* sv = sn + (size_t)s * m;
    double* gv = g + (size_t)s * (m + 1);
    for (int i = 0; i <= j; ++i) hc[i] = gg[i] + gg[m + 1 + i];
    hc[j + 1] = sqrt(gg[2 * (m + 1)]);
    for (int i = 0; i < j; ++i) {
      const double a = c[i] * hc[i] + sv[i] * hc[i + 1];
      hc[i + 1] = -sv[i] * hc[i] + c[i] * hc[i + 1];
      hc[i] = a;
    }
    const double rr = hypot(hc[j], hc[j + 1]);
    c[j] = rr > 0.0 ? hc[j] / rr : 1.0;
    sv[j] = rr > 0.0 ? hc[j + 1] / rr : 0.0;
    hc[j] = rr;
    hc[j + 1] = 0.0;
    gv[j + 1] = -sv[j] * gv[j];
    gv[j] = c[j] * gv[j];
    const int it = iters[s] + 1;
    iters[s] = it;
    kk[s] = j + 1;
    const double est = fabs(gv[j + 1]);
    if (!(est > tol[s]) || it >= maxit || j + 1 >= m) act[s] = 0;
    else live += 1.0;
  }
  const double n = block_sum256(live, sh);
  if (threadIdx.x == 0) {
    nact[j] = (int)n;
    __threadfence_system();
    *jp = j + 1;
  }
}

// y_s = H_s(0:k,0:k)^{-1} g_s(0:k), k = kk[s], for the scenes of the cycle (one thread per scene)
__global__ void k_seg_backsolve(int ns, int m, const int* __restrict__ cyc, const int* __restrict__ kk,
                                const double* __restrict__ H, const double* __restrict__ g, double* y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns || !cyc[s]) return;
  const int k = kk[s];
  const double* Hs = H + (size_t)s * (m + 1) * m;
  const double* gs = g + (size_t)s * (m + 1);
  double* ys = y + (size_t)s * m;
  for (int i = k - 1; i >= 0; --i) {
    double a = gs[i];
    for (int jj = i + 1; jj < k; ++jj) a -= Hs[(size_t)(m + 1) * jj + i] * ys[jj];
    const double d = Hs[(size_t)(m + 1) * i + i];
    ys[i] = d != 0.0 ? a / d : 0.0;
  }
}

// x += sum_{k < kk[s]} y_s[k] Z_k on the tiles of the cycle's scenes (flexible GMRES update)
__global__ void __launch_bounds__(256) k_seg_combine(SegTiles T, const double* __restrict__ Z, long ld, int m,
                                                     const int* __restrict__ cyc, const int* __restrict__ kk,
                                                     const double* __restrict__ y, double* __restrict__ x) {
  const int t = blockIdx.x, s = T.scene[t];
  if (!cyc[s]) return;
  const int k = kk[s];
  if (k == 0) return;
  __shared__ double c[kMaxRestart];
  for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = y[(size_t)s * m + i];
  __syncthreads();
  for (int i = T.beg[t] + (int)threadIdx.x; i < T.end[t]; i += blockDim.x) {
    double acc = x[i];
    for (int q = 0; q < k; ++q) acc += c[q] * Z[(size_t)q * ld + i];
    x[i] = acc;
  }
}

// r = b - w on the tiles of the scenes with mask[s]
__global__ void __launch_bounds__(256) k_seg_resid(SegTiles T, const double* __restrict__ b,
                                                   const double* __restrict__ w, const int* __restrict__ mask,
                                                   double* __restrict__ r) {
  const int t = blockIdx.x, s = T.scene[t];
  if (!mask[s]) return;
  for (int i = T.beg[t] + (int)threadIdx.x; i < T.end[t]; i += blockDim.x) r[i] = b[i] - w[i];
}

// End of a cycle (or the start, first = 1): beta_s = |r_s| from rr[s] for the scenes of the cycle.
// On the first call bnorm[s] = beta_s and tol[s] = rtol beta_s.  A scene is done once beta_s <=
// tol[s], once it has maxit iterations, or when beta_s is not finite (FLAG_NONFINITE); the others
// start a new cycle (act = cyc = 1, kk = 0, g = beta e_1).  One block; the number of scenes not done
// goes to the host-mapped *notdone and *jp = 0.
__global__ void __launch_bounds__(256) k_seg_restart(int ns, int m, int first, int* cyc, int* act, int* done, int* kk,
                                                     const int* __restrict__ iters, int maxit,
                                                     const double* __restrict__ rr, double* bnorm, double* tol,
                                                     double rtol, double* relres, double* g, int* jp, int* flags,
                                                     volatile int* notdone) {
  __shared__ double sh[8];
  double live = 0.0;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    if (!cyc[s]) continue;
    const double beta = sqrt(rr[s]);
    if (first) {
      bnorm[s] = beta;
      tol[s] = rtol * beta;
    }
    relres[s] = bnorm[s] > 0.0 ? beta / bnorm[s] : 0.0;
    const bool fin = isfinite(beta);
    if (!fin) atomicExch(&flags[FLAG_NONFINITE], 1);
    const bool stop = !fin || !(beta > tol[s]) || iters[s] >= maxit;
    done[s] = stop ? 1 : 0;
    act[s] = cyc[s] = stop ? 0 : 1;
    kk[s] = 0;
    if (!stop) {
      double* gv = g + (size_t)s * (m + 1);
      gv[0] = beta;
      for (int i = 1; i <= m; ++i) gv[i] = 0.0;
      live += 1.0;
    }
  }
  const double n = block_sum256(live, sh);
  if (threadIdx.x == 0) {
    *notdone = (int)n;
    __threadfence_system();
    *jp = 0;
  }
}

// V_0 = r / beta_s (beta_s = g[s][0]) on the tiles of the active scenes
__global__ void __launch_bounds__(256) k_seg_start(SegTiles T, const double* __restrict__ r,
                                                   const int* __restrict__ act, const double* __restrict__ g, int m,
                                                   double* __restrict__ V) {
  const int t = blockIdx.x, s = T.scene[t];
  if (!act[s]) return;
  const double inv = 1.0 / g[(size_t)s * (m + 1)];
  for (int i = T.beg[t] + (int)threadIdx.x; i < T.end[t]; i += blockDim.x) V[i] = r[i] * inv;
}

__global__ void k_seg_init(int ns, int* cyc, int* done, int* iters) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  cyc[s] = 1;
  done[s] = 0;
  iters[s] = 0;
}

// Table-driven copies between a batch's per-scene arrays and the union's: entry e copies cnt[e]
// elements from src[e] to dst[e], one block per entry.
__global__ void k_gather_f64(int nent, const double* const* __restrict__ src, double* const* __restrict__ dst,
                             const int64_t* __restrict__ cnt) {
  const int e = blockIdx.x;
  if (e >= nent) return;
  const double* a = src[e];
  double* b = dst[e];
  const int64_t n = cnt[e];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b[i] = a[i];
}
// int32 copy with an additive offset (vertex and region ids of a batch), one block per entry
__global__ void k_gather_ids(int nent, const int32_t* const* __restrict__ src, int32_t* const* __restrict__ dst,
                             const int64_t* __restrict__ cnt, const int32_t* __restrict__ add) {
  const int e = blockIdx.x;
  if (e >= nent) return;
  const int32_t* a = src[e];
  int32_t* b = dst[e];
  const int64_t n = cnt[e];
  const int32_t o = add[e];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b[i] = (a ? a[i] : 0) + o;  // no source: the offset alone
}
// Contact c of a batch call belongs to the scene s with coff[s] <= c < coff[s+1]; its (offset) vertex
// id must lie in [voff[s], voff[s+1]) and its (offset) region in [roff[s], roff[s+1]), else
// FLAG_BADINDEX.
__global__ void k_check_batch_ids(int nc, const int32_t* __restrict__ vertex, const int32_t* __restrict__ region,
                                  int ns, const int32_t* __restrict__ coff, const int32_t* __restrict__ voff,
                                  const int32_t* __restrict__ roff, int* flags) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  int lo = 0, hi = ns - 1;  // last s with coff[s] <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (coff[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  const int v = vertex[c];
  bool bad = v < voff[lo] || v >= voff[lo + 1];
  if (region) bad = bad || region[c] < roff[lo] || region[c] >= roff[lo + 1];
  if (bad) atomicExch(&flags[FLAG_BADINDEX], 1);
}
// FP32 copy (per-tet activation gradients)
__global__ void k_gather_f32(int nent, const float* const* __restrict__ src, float* const* __restrict__ dst,
                                const int64_t* __restrict__ cnt) {
  const int e = blockIdx.x;
  if (e >= nent) return;
  const float* a = src[e];
  float* b = dst[e];
  const int64_t n = cnt[e];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) b[i] = a[i];
}

}  // namespace

void launch_seg_dot_step(const SegTiles& T, const double* V, long ld, const int* jp, int m, bool self, const int* act,
                         double* partial, unsigned* cnt, int K, double* gsb, int gstride, int goff, cudaStream_t s) {
  g_launches += 1;
  k_seg_dot_step<<<dim3(T.n, self ? 1 : m), 256, 0, s>>>(T, V, ld, jp, m, self ? 1 : 0, act, partial, cnt, K, gsb,
                                                          gstride, goff);
}
void launch_seg_sq(const SegTiles& T, const double* x, const int* mask, double* partial, unsigned* cnt, int K, int slot,
                   double* out, cudaStream_t s) {
  g_launches += 1;
  k_seg_sq<<<T.n, 256, 0, s>>>(T, x, mask, partial, cnt, K, slot, out);
}
void launch_seg_axpy_step(const SegTiles& T, double* V, long ld, const int* jp, int m, const int* act,
                          const double* gsb, int gstride, int goff, cudaStream_t s) {
  g_launches += 1;
  k_seg_axpy_step<<<T.n, 256, 0, s>>>(T, V, ld, jp, m, act, gsb, gstride, goff);
}
void launch_seg_normalize_step(const SegTiles& T, double* V, long ld, const int* jp, int m, const int* act,
                               const double* gsb, int gstride, int noff, cudaStream_t s) {
  g_launches += 1;
  k_seg_normalize_step<<<T.n, 256, 0, s>>>(T, V, ld, jp, m, act, gsb, gstride, noff);
}
void launch_seg_copy_step(const SegTiles& T, const double* src, bool src_idx, double* dst, bool dst_idx, long ld,
                          const int* jp, int m, const int* act, const double* d, cudaStream_t s, float2* split) {
  g_launches += 1;
  k_seg_copy_step<<<T.n, 256, 0, s>>>(T, src, src_idx ? 1 : 0, dst, dst_idx ? 1 : 0, ld, jp, m, act, d, split);
}
void launch_seg_givens(int ns, int* jp, int m, int* act, const double* gsb, int gstride, double* H, double* cs,
                       double* sn, double* g, int* kk, int* iters, const double* tol, int maxit, int* nact,
                       cudaStream_t s) {
  g_launches += 1;
  k_seg_givens<<<1, 256, 0, s>>>(ns, jp, m, act, gsb, gstride, H, cs, sn, g, kk, iters, tol, maxit, nact);
}
void launch_seg_backsolve(int ns, int m, const int* cyc, const int* kk, const double* H, const double* g, double* y,
                          cudaStream_t s) {
  g_launches += 1;
  k_seg_backsolve<<<nblk(ns, 128), 128, 0, s>>>(ns, m, cyc, kk, H, g, y);
}
void launch_seg_combine(const SegTiles& T, const double* Z, long ld, int m, const int* cyc, const int* kk,
                        const double* y, double* x, cudaStream_t s) {
  g_launches += 1;
  k_seg_combine<<<T.n, 256, 0, s>>>(T, Z, ld, m, cyc, kk, y, x);
}
void launch_seg_resid(const SegTiles& T, const double* b, const double* w, const int* mask, double* r,
                      cudaStream_t s) {
  g_launches += 1;
  k_seg_resid<<<T.n, 256, 0, s>>>(T, b, w, mask, r);
}
void launch_seg_restart(int ns, int m, bool first, int* cyc, int* act, int* done, int* kk, const int* iters,
                        int maxit, const double* rr, double* bnorm, double* tol, double rtol, double* relres,
                        double* g, int* jp, int* flags, int* notdone, cudaStream_t s) {
  g_launches += 1;
  k_seg_restart<<<1, 256, 0, s>>>(ns, m, first ? 1 : 0, cyc, act, done, kk, iters, maxit, rr, bnorm, tol, rtol,
                                  relres, g, jp, flags, notdone);
}
void launch_seg_start(const SegTiles& T, const double* r, const int* act, const double* g, int m, double* V,
                      cudaStream_t s) {
  g_launches += 1;
  k_seg_start<<<T.n, 256, 0, s>>>(T, r, act, g, m, V);
}
void launch_seg_init(int ns, int* cyc, int* done, int* iters, cudaStream_t s) {
  g_launches += 1;
  k_seg_init<<<nblk(ns, 128), 128, 0, s>>>(ns, cyc, done, iters);
}
void launch_gather_f64(int nent, const double* const* src, double* const* dst, const int64_t* cnt, cudaStream_t s) {
  if (nent <= 0) return;
  g_launches += 1;
  k_gather_f64<<<nent, 256, 0, s>>>(nent, src, dst, cnt);
}
void launch_gather_ids(int nent, const int32_t* const* src, int32_t* const* dst, const int64_t* cnt,
                       const int32_t* add, cudaStream_t s) {
  if (nent <= 0) return;
  g_launches += 1;
  k_gather_ids<<<nent, 256, 0, s>>>(nent, src, dst, cnt, add);
}
void launch_check_batch_ids(int nc, const int32_t* vertex, const int32_t* region, int ns, const int32_t* coff,
                            const int32_t* voff, const int32_t* roff, int* flags, cudaStream_t s) {
  if (nc <= 0) return;
  g_launches += 1;
  k_check_batch_ids<<<nblk(nc, 128), 128, 0, s>>>(nc, vertex, region, ns, coff, voff, roff, flags);
}
void launch_gather_f32(int nent, const float* const* src, float* const* dst, const int64_t* cnt, cudaStream_t s) {
  if (nent <= 0) return;
  g_launches += 1;
  k_gather_f32<<<nent, 256, 0, s>>>(nent, src, dst, cnt);
}

}  // namespace ncpadj
