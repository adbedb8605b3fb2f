// Sparse and dense linear algebra of the adjoint solve.
//
//  * block sparse matrix-vector product with the assembled script_A^T (3x3 blocks),
//  * A^{-1} x = P^T S^T S P x through the explicit sparse inverse S = L^{-1} of the scalar
//    elastic factor, applied to the 3 coordinates at once (Sec. 3, sparse-inverse factorisation);
//    the rows of S are contiguous column ranges (postordered elimination tree), those of S^T the
//    elimination-tree paths,
//  * the contact-space pieces of the Woodbury preconditioner (Eq. woodbury_formula, used in the
//    form without K^{-1}): Delassus entries (A_s^{-1})_{v_a v_b}, the capacitance
//    C = I + h^2 K^T D, its inverse by in-place Gauss-Jordan elimination with partial pivoting in
//    one cooperative launch, and the gather/scatter with the contact frames,
//  * the vector kernels of CG and restarted GMRES (Sec. 4.4).
#include <math.h>

#include <cooperative_groups.h>

#include "dfloat.cuh"
#include "kernels.cuh"

namespace ncpadj {

thread_local long long g_launches = 0;

namespace {

inline int nblk(long n, int b) { return (int)((n + b - 1) / b); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Half a warp per vertex row: lane l of the half takes blocks rp[v] + l, rp[v] + l + 16, ... and the
// three row sums are reduced over the half-warp (the row-per-thread form left the GPU nearly empty:
// one thread per scalar row, each walking its ~15 blocks with dependent loads).
// jp (nullable): y is written at y + (*jp + 1) * yld (the next Arnoldi vector of a captured step)
template <typename V>
__global__ void __launch_bounds__(256) k_bsr_spmv_hw(int nv, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const V* __restrict__ val,
                                                     const double* __restrict__ x, double* __restrict__ y,
                                                     const int* __restrict__ jp = nullptr, long yld = 0,
                                                     Mask mk = Mask{}) {
  if (jp) y += (size_t)(*jp + 1) * yld;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = t >> 4, l = t & 15;
  // rows of scenes outside the mask are skipped (not returned: the half-warps share shuffles)
  const bool live = v < nv && mk.on(v);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  if (live) {
    const int pe = rp[v + 1];
    for (int p = rp[v] + l; p < pe; p += 16) {
      const int c = col[p];
      const V* B = val + 9 * (size_t)p;
      const double x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
      a0 += (double)B[0] * x0 + (double)B[1] * x1 + (double)B[2] * x2;
      a1 += (double)B[3] * x0 + (double)B[4] * x1 + (double)B[5] * x2;
      a2 += (double)B[6] * x0 + (double)B[7] * x1 + (double)B[8] * x2;
    }
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (live && l == 0) {
    y[3 * (size_t)v] = a0;
    y[3 * (size_t)v + 1] = a1;
    y[3 * (size_t)v + 2] = a2;
  }
}

// The same product for FP32 block values with x given as double-float pairs x2 = (hi, lo): every
// product and sum in double-float on the FP32 pipes (about 48 significant bits, FP64-class
// accuracy), y in FP64.  The FP64 accumulation above spends 9 FMAs and 9 conversions per block
// on this part's slow FP64 pipe, which bounds that kernel far below the memory rate.
__global__ void __launch_bounds__(256) k_bsr_spmv_ff(int nv, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, const float* __restrict__ val,
                                                     const float2* __restrict__ x2, double* __restrict__ y,
                                                     const int* __restrict__ jp, long yld, Mask mk) {
  if (jp) y += (size_t)(*jp + 1) * yld;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = t >> 4, l = t & 15;
  const bool live = v < nv && mk.on(v);  // skipped, not returned: the half-warps share shuffles
  float h0 = 0.f, h1 = 0.f, h2 = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f;
  if (live) {
    const int pe = rp[v + 1];
    for (int p = rp[v] + l; p < pe; p += 16) {
      const int c = col[p];
      const float* B = val + 9 * (size_t)p;
      const float2 a = x2[3 * (size_t)c], b = x2[3 * (size_t)c + 1], d = x2[3 * (size_t)c + 2];
      df_fma(B[0], a.x, a.y, h0, l0);
      df_fma(B[1], b.x, b.y, h0, l0);
      df_fma(B[2], d.x, d.y, h0, l0);
      df_fma(B[3], a.x, a.y, h1, l1);
      df_fma(B[4], b.x, b.y, h1, l1);
      df_fma(B[5], d.x, d.y, h1, l1);
      df_fma(B[6], a.x, a.y, h2, l2);
      df_fma(B[7], b.x, b.y, h2, l2);
      df_fma(B[8], d.x, d.y, h2, l2);
    }
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const float a0 = __shfl_xor_sync(0xffffffffu, h0, o), b0 = __shfl_xor_sync(0xffffffffu, l0, o);
    const float a1 = __shfl_xor_sync(0xffffffffu, h1, o), b1 = __shfl_xor_sync(0xffffffffu, l1, o);
    const float a2 = __shfl_xor_sync(0xffffffffu, h2, o), b2 = __shfl_xor_sync(0xffffffffu, l2, o);
    df_add(h0, l0, a0, b0);
    df_add(h1, l1, a1, b1);
    df_add(h2, l2, a2, b2);
  }
  if (live && l == 0) {
    y[3 * (size_t)v] = df_to_double(h0, l0);
    y[3 * (size_t)v + 1] = df_to_double(h1, l1);
    y[3 * (size_t)v + 2] = df_to_double(h2, l2);
  }
}

// x2[i] = (hi, lo) of x[i]: the double-float input of k_bsr_spmv_ff
__global__ void k_split(int n, const double* __restrict__ x, float2* __restrict__ x2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x2[i] = df_split(x[i]);
}

// x[k] = sum_j B[piv[k]][j] y[piv[j]]: the Gauss-Jordan result B applied to y with both permutations.
// A block stages y[piv[.]] (as T) in shared memory, then two warps per row split the columns, each
// lane with four independent accumulators; T = float accumulates in FP32 (preconditioner apply).
template <typename T>
__global__ void __launch_bounds__(256) k_cap_apply(int n, const T* __restrict__ B, const int32_t* __restrict__ piv,
                                                   const double* __restrict__ y, double* __restrict__ x,
                                                   const int* __restrict__ act = nullptr, int scene = 0) {
  if (act && !act[scene]) return;  // the block's scene is idle (uniform over the launch)
  extern __shared__ __align__(16) unsigned char smraw[];
  T* ys = reinterpret_cast<T*>(smraw);
  __shared__ T part[4][2];
  for (int j = threadIdx.x; j < n; j += blockDim.x) ys[j] = (T)y[piv[j]];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rloc = warp >> 1, half = warp & 1;
  const int k = blockIdx.x * 4 + rloc;
  T acc = 0;
  if (k < n) {
    const T* row = B + (size_t)piv[k] * n;
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int j = half * 32 + lane;
    for (; j + 192 < n; j += 256) {
      a0 += row[j] * ys[j];
      a1 += row[j + 64] * ys[j + 64];
      a2 += row[j + 128] * ys[j + 128];
      a3 += row[j + 192] * ys[j + 192];
    }
    for (; j < n; j += 64) a0 += row[j] * ys[j];
    acc = (a0 + a1) + (a2 + a3);
  }
  acc = warp_sum(acc);
  if (lane == 0) part[rloc][half] = acc;
  __syncthreads();
  if (threadIdx.x < 4) {
    const int kk = blockIdx.x * 4 + threadIdx.x;
    if (kk < n) x[kk] = (double)(part[threadIdx.x][0] + part[threadIdx.x][1]);
  }
}

__global__ void k_diag_inv(int nv, const int32_t* diag_slot, const double* val, const float* val32, double* dinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nv) return;
  const int v = i / 3, r = i - 3 * v;
  const size_t k = 9 * (size_t)diag_slot[v] + 4 * r;
  dinv[i] = 1.0 / (val ? val[k] : (double)val32[k]);
}

// Chunked product of a CSR matrix with 3 right-hand sides: chunk k covers entries
// [cbeg[k], cend[k]) of row crow[k] (at most 32 PL), one warp per chunk with PL loads in flight per
// lane; partial sums are added atomically into y[3 out(row) + r] (y zeroed by the caller),
// out(row) = omap ? omap[row] : row.  Splitting the long rows near the elimination-tree root over
// many warps keeps the product bandwidth- rather than latency-bound.
// jp (nullable): x is taken at x + (*jp) * xld -- the step index of a captured GMRES step
template <typename V, typename X, typename Y, typename Acc = Y, int PL = 8>
__global__ void __launch_bounds__(256) k_spmv_chunks(int nchunks, const int32_t* __restrict__ crow,
                                                     const int64_t* __restrict__ cbeg, const int64_t* __restrict__ cend,
                                                     const int32_t* __restrict__ col, const V* __restrict__ val,
                                                     const int32_t* __restrict__ omap, const X* __restrict__ x,
                                                     Y* __restrict__ y, const int* __restrict__ jp = nullptr,
                                                     long xld = 0, Mask mk = Mask{}) {
  if (jp) x += (size_t)(*jp) * xld;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nchunks) return;
  if (!mk.on(crow[k])) return;  // whole warp: one chunk per warp (positions keep their scene)
  const int64_t b = cbeg[k], e = cend[k];
  Acc a0 = 0, a1 = 0, a2 = 0;
  int c[PL];
  V s[PL];
#pragma unroll
  for (int u = 0; u < PL; ++u) {
    const int64_t p = b + lane + 32 * u;
    c[u] = (p < e) ? col[p] : -1;
    s[u] = (p < e) ? val[p] : V(0);
  }
#pragma unroll
  for (int u = 0; u < PL; ++u)
    if (c[u] >= 0) {
      a0 += (Acc)s[u] * (Acc)x[3 * c[u]];
      a1 += (Acc)s[u] * (Acc)x[3 * c[u] + 1];
      a2 += (Acc)s[u] * (Acc)x[3 * c[u] + 2];
    }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  if (lane == 0) {
    const int row = crow[k];
    const int o = omap ? omap[row] : row;
    atomicAdd(&y[3 * o], (Y)a0);
    atomicAdd(&y[3 * o + 1], (Y)a1);
    atomicAdd(&y[3 * o + 2], (Y)a2);
  }
}

// The product with S = L^{-1} in a postordered elimination tree: row i of S holds exactly the
// descendants of i, the contiguous column range [i - size(i) + 1, i], so no column index is stored.
// Chunk k covers entries [cbeg[k], cend[k]) of row crow[k] (at most 32 PL), whose columns run from
// c0[k] upwards; one warp per chunk, PL values per lane in flight, x read contiguously; partial sums added
// atomically into y[3 row + r] (y zeroed by the caller).
template <typename V, typename X, typename Y, typename Acc = Y, int PL = 8>
__global__ void __launch_bounds__(256) k_spmv_range_chunks(int nchunks, const int32_t* __restrict__ crow,
                                                           const int64_t* __restrict__ cbeg,
                                                           const int64_t* __restrict__ cend,
                                                           const int32_t* __restrict__ c0, const V* __restrict__ val,
                                                           const X* __restrict__ x, Y* __restrict__ y,
                                                           Mask mk = Mask{}) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nchunks) return;
  const int row = crow[k];
  if (!mk.on(row)) return;  // whole warp: one chunk per warp (positions keep their scene)
  const int64_t b = cbeg[k], e = cend[k];
  const int col0 = c0[k];
  Acc a0 = 0, a1 = 0, a2 = 0;
  V s[PL];
#pragma unroll
  for (int u = 0; u < PL; ++u) {
    const int64_t p = b + lane + 32 * u;
    s[u] = (p < e) ? val[p] : V(0);
  }
#pragma unroll
  for (int u = 0; u < PL; ++u) {
    const int off = lane + 32 * u;
    if (b + off < e) {
      const size_t c = 3 * (size_t)(col0 + off);
      a0 += (Acc)s[u] * (Acc)x[c];
      a1 += (Acc)s[u] * (Acc)x[c + 1];
      a2 += (Acc)s[u] * (Acc)x[c + 2];
    }
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  if (lane == 0) {
    atomicAdd(&y[3 * row], (Y)a0);
    atomicAdd(&y[3 * row + 1], (Y)a1);
    atomicAdd(&y[3 * row + 2], (Y)a2);
  }
}

// out[3p + r] = x[3 perm[p] + r] (x taken at x + (*jp) * ld when jp is given): the input of the
// product with S, whose columns are elimination positions
template <typename O>
__global__ void k_to_position(int nv, const double* __restrict__ x, const int* __restrict__ jp, long ld,
                              const int32_t* __restrict__ perm, O* __restrict__ out, Mask mk = Mask{}) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nv) return;
  if (jp) x += (size_t)(*jp) * ld;
  const int p = i / 3, r = i - 3 * p;
  if (!mk.on(p)) return;
  out[i] = (O)x[3 * (size_t)perm[p] + r];
}

// Contact rows of A^{-1} x from w = S P x: (A^{-1} x)_v = sum_i S[i][p(v)] w_i, and column p(v) of S
// (row p(v) of S^T) lives on the elimination-tree path from p(v) to the root.  One warp per
// contact walks that path; the result u_c is turned into s_c = K'_c F_c u_c at once (K' = K^T for
// the adjoint), the input of the capacitance solve.
template <typename V, typename W>
__global__ void __launch_bounds__(256) k_path_gather(int nc, const int32_t* __restrict__ cvertex,
                                                     const int32_t* __restrict__ iperm, const int64_t* __restrict__ ptr,
                                                     const int32_t* __restrict__ col, const V* __restrict__ val,
                                                     const W* __restrict__ w, const double* __restrict__ frame,
                                                     const double* __restrict__ cdata, int transpose,
                                                     double* __restrict__ sc, Mask mk = Mask{}) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nc) return;
  if (!mk.on(cvertex[c])) return;  // whole warp: one contact per warp
  const int pv = iperm[cvertex[c]];
  const int64_t b = ptr[pv], e = ptr[pv + 1];
  double u0 = 0.0, u1 = 0.0, u2 = 0.0;
  // 8 entries per lane in flight (index and value first, then the gathers), 256 per round
  for (int64_t p0 = b; p0 < e; p0 += 256) {
    int ci[8];
    double sv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t p = p0 + lane + 32 * k;
      ci[k] = p < e ? col[p] : -1;
      sv[k] = p < e ? (double)val[p] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (ci[k] >= 0) {
        u0 += sv[k] * (double)w[3 * (size_t)ci[k]];
        u1 += sv[k] * (double)w[3 * (size_t)ci[k] + 1];
        u2 += sv[k] * (double)w[3 * (size_t)ci[k] + 2];
      }
  }
  u0 = warp_sum(u0);
  u1 = warp_sum(u1);
  u2 = warp_sum(u2);
  if (lane == 0) {
    const double* F = frame + 9 * (size_t)c;
    const double* K = cdata + 12 * (size_t)c;
    double y[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = F[3 * i] * u0 + F[3 * i + 1] * u1 + F[3 * i + 2] * u2;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      sc[3 * c + j] = transpose ? K[j] * y[0] + K[3 + j] * y[1] + K[6 + j] * y[2]
                                : K[3 * j] * y[0] + K[3 * j + 1] * y[1] + K[3 * j + 2] * y[2];
  }
}

// w += coef S P J^T t: contact c's force F_c^T t_c at vertex v_c enters S P x through column p(v_c)
// of S, i.e. along the elimination-tree path of p(v_c) (one warp per contact, atomics).
template <typename V, typename W>
__global__ void __launch_bounds__(256) k_path_scatter(int nc, const int32_t* __restrict__ cvertex,
                                                      const int32_t* __restrict__ iperm, const int64_t* __restrict__ ptr,
                                                      const int32_t* __restrict__ col, const V* __restrict__ val,
                                                      const double* __restrict__ frame, const double* __restrict__ t,
                                                      double coef, W* w, Mask mk = Mask{}) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nc) return;
  if (!mk.on(cvertex[c])) return;  // whole warp: one contact per warp
  const double* F = frame + 9 * (size_t)c;
  const double t0 = t[3 * c], t1 = t[3 * c + 1], t2 = t[3 * c + 2];
  const double f0 = coef * (F[0] * t0 + F[3] * t1 + F[6] * t2);
  const double f1 = coef * (F[1] * t0 + F[4] * t1 + F[7] * t2);
  const double f2 = coef * (F[2] * t0 + F[5] * t1 + F[8] * t2);
  const int pv = iperm[cvertex[c]];
  const int64_t b = ptr[pv], e = ptr[pv + 1];
  for (int64_t p0 = b; p0 < e; p0 += 256) {
    int ci[8];
    double sv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t p = p0 + lane + 32 * k;
      ci[k] = p < e ? col[p] : -1;
      sv[k] = p < e ? (double)val[p] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (ci[k] >= 0) {
        atomicAdd(&w[3 * (size_t)ci[k]], (W)(sv[k] * f0));
        atomicAdd(&w[3 * (size_t)ci[k] + 1], (W)(sv[k] * f1));
        atomicAdd(&w[3 * (size_t)ci[k] + 2], (W)(sv[k] * f2));
      }
  }
}

// Ds[a][b] = sum_k S[k][ia] S[k][ib]: rows ia, ib of S^T are the elimination-tree paths of
// ia and ib; they share exactly the path from their lowest common ancestor to the root, which
// is a common suffix of both rows.
__global__ void k_delassus(int nc, const int32_t* __restrict__ cvertex, const int32_t* __restrict__ iperm,
                           const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, double* Ds) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)nc * nc) return;
  const int a = (int)(idx / nc), b = (int)(idx - (long)a * nc);
  const int ia = iperm[cvertex[a]], ib = iperm[cvertex[b]];
  int64_t pa = ptr[ia + 1] - 1, pb = ptr[ib + 1] - 1;
  const int64_t ea = ptr[ia], eb = ptr[ib];
  double acc = 0.0;
  while (pa >= ea && pb >= eb && col[pa] == col[pb]) {
    acc += val[pa] * val[pb];
    --pa;
    --pb;
  }
  Ds[idx] = acc;
}

// score_c = h^2 |K_c|_F (A_s^{-1})_{v_c v_c}: how far contact c's rows of the capacitance
// I + h^2 K^T D stand from the identity.  (A_s^{-1})_{vv} = |S[:, p(v)]|^2 is the squared norm of row
// p(v) of S^T (the elimination-tree path of v's position); one warp per contact.
__global__ void k_contact_score(int nc, const int32_t* __restrict__ cvertex, const int32_t* __restrict__ iperm,
                                const int64_t* __restrict__ ptr, const double* __restrict__ val,
                                const double* __restrict__ cdata, double h2, double* __restrict__ score) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nc) return;
  const int pv = iperm[cvertex[c]];
  double acc = 0.0;
  for (int64_t p = ptr[pv] + lane; p < ptr[pv + 1]; p += 32) acc += val[p] * val[p];
  acc = warp_sum(acc);
  if (lane == 0) {
    const double* K = cdata + 12 * (size_t)c;
    double kk = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) kk += K[i] * K[i];
    score[c] = h2 * sqrt(kk) * acc;
  }
}

// the contacts idx[0..nk) of the capacitance set, copied together: vertex, frame (9), K and k_mu (12)
__global__ void k_gather_contacts(int nk, const int32_t* __restrict__ idx, const int32_t* __restrict__ vertex,
                                  const double* __restrict__ frame, const double* __restrict__ cdata,
                                  int32_t* __restrict__ ov, double* __restrict__ of, double* __restrict__ oc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const int c = idx[k];
  ov[k] = vertex[c];
#pragma unroll
  for (int i = 0; i < 9; ++i) of[9 * (size_t)k + i] = frame[9 * (size_t)c + i];
#pragma unroll
  for (int i = 0; i < 12; ++i) oc[12 * (size_t)k + i] = cdata[12 * (size_t)c + i];
}

// Single-vertex bilateral bindings as members of the capacitance set: binding b acts on vertex[b]
// through J_b = e_v^T (x) I_3 with the stiffness I / E_b, i.e. a vertex "contact" with the identity
// frame and K = I / E_b (no friction coefficient).  Written after the first `off` candidates.
__global__ void k_binding_capdata(int nb, const int32_t* __restrict__ vertex, const double* __restrict__ compliance,
                                  int off, int32_t* __restrict__ ov, double* __restrict__ of,
                                  double* __restrict__ oc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const size_t k = (size_t)off + b;
  ov[k] = vertex[b];
  const double kb = 1.0 / compliance[b];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    of[9 * k + i] = (i % 4 == 0) ? 1.0 : 0.0;
    oc[12 * k + i] = (i % 4 == 0) ? kb : 0.0;
  }
#pragma unroll
  for (int i = 9; i < 12; ++i) oc[12 * k + i] = 0.0;
}

// C[3a+r][3b+s] = delta + h^2 Ds[a][b] sum_l K'_a[r][l] (F_a F_b^T)[l][s],  K' = K^T (adjoint) or K
__global__ void k_cap_form(int nc, const double* __restrict__ Ds, const double* __restrict__ frame,
                           const double* __restrict__ cdata, double h2, int transpose, double* C) {
  const long n = 3L * nc;
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int R = (int)(idx / n), Cc = (int)(idx - (long)R * n);
  const int a = R / 3, r = R - 3 * a, b = Cc / 3, s = Cc - 3 * b;
  const double* Fa = frame + 9 * (size_t)a;
  const double* Fb = frame + 9 * (size_t)b;
  const double* Ka = cdata + 12 * (size_t)a;
  double acc = 0.0;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const double ff = Fa[3 * l] * Fb[3 * s] + Fa[3 * l + 1] * Fb[3 * s + 1] + Fa[3 * l + 2] * Fb[3 * s + 2];
    acc += (transpose ? Ka[3 * l + r] : Ka[3 * r + l]) * ff;
  }
  C[idx] = (R == Cc ? 1.0 : 0.0) + h2 * Ds[(size_t)a * nc + b] * acc;
}

// ---- vector kernels of the Krylov solves -----------------------------------------------

__global__ void k_axpby(int n, double a, const double* x, double b, const double* y, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * (y ? y[i] : 0.0);
}
__global__ void k_rhs(int n, const double* dq, const double* dv, double inv_h, double* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = dq[i] + (dv ? dv[i] * inv_h : 0.0);
}
__global__ void k_mul(int n, const double* a, const double* b, double* y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] * b[i];
}

// partial[k][blk] = sum over this block's slice of V_k . w
// out[k] = V_k . w in one launch: every block writes its partial for vector k (blockIdx.y), and the
// last block to finish (counted in cnt[k], which it resets) reduces the partials in a fixed order.
__global__ void k_multi_dot_fused(int n, const double* __restrict__ V, long ld, const double* __restrict__ w,
                                  double* partial, unsigned* cnt, double* out) {
  const int k = blockIdx.y;
  const double* vk = V + (size_t)k * ld;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    acc += vk[i] * w[i];
  acc = warp_sum(acc);
  __shared__ double sh[32];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      partial[(size_t)k * gridDim.x + blockIdx.x] = v;
      __threadfence();
      last = atomicAdd(&cnt[k], 1u) == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(&partial[(size_t)k * gridDim.x + i]);
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    out[k] = r;
    cnt[k] = 0;
  }
}

// Step-indexed Gram-Schmidt kernels of a captured GMRES step: j = *jp, the new vector is
// V_{j+1} = V + (j + 1) ld and the basis so far is V_0..V_j.
// out[k] = V_k . V_{j+1} for k <= j (blockIdx.y = k; columns above j return at once); with self,
// out[0] = V_{j+1} . V_{j+1}.
__global__ void k_multi_dot_idx(int n, const double* __restrict__ V, long ld, const int* __restrict__ jp, int self,
                                double* partial, unsigned* cnt, double* out) {
  const int j = *jp;
  const int k = blockIdx.y;
  if (k > (self ? 0 : j)) return;
  const double* w = V + (size_t)(j + 1) * ld;
  const double* vk = self ? w : V + (size_t)k * ld;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    acc += vk[i] * w[i];
  acc = warp_sum(acc);
  __shared__ double sh[32];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      partial[(size_t)k * gridDim.x + blockIdx.x] = v;
      __threadfence();
      last = atomicAdd(&cnt[k], 1u) == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(&partial[(size_t)k * gridDim.x + i]);
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    out[k] = r;
    cnt[k] = 0;
  }
}
// V_{j+1} -= sum_{k <= j} coef[k] V_k
// 256 threads per block = 32 elements x 8 groups of the basis: thread (e, g) sums coef[k] V_k[i] over
// k = g, g + 8, ..., and the eight partial sums of an element are added in group order.
__global__ void __launch_bounds__(256) k_multi_axpy_idx(int n, const double* __restrict__ V, long ld,
                                                        const int* __restrict__ jp, const double* __restrict__ coef,
                                                        double* __restrict__ Vw) {
  const int j = *jp;
  const int e = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + e;
  __shared__ double part[8][32];
  double acc = 0.0;
  if (i < n)
    for (int k = g; k <= j; k += 8) acc += coef[k] * V[(size_t)k * ld + i];
  part[g][e] = acc;
  __syncthreads();
  if (g == 0 && i < n) {
    double t = part[0][e];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += part[q][e];
    double* w = Vw + (size_t)(j + 1) * ld;
    w[i] -= t;
  }
}
// V_{j+1} /= sqrt(*nrm2); h_slot = the norm
__global__ void k_normalize_idx(int n, double* V, long ld, const int* __restrict__ jp, const double* nrm2,
                                double* h_slot) {
  const int j = *jp;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double nr = sqrt(*nrm2);
  double* v = V + (size_t)(j + 1) * ld;
  if (i < n) v[i] = (nr > 0.0) ? v[i] / nr : 0.0;
  if (i == 0) *h_slot = nr;
}
// Y_j = x with j = *jp read on the device (column j of Y, stride ld)
__global__ void k_copy_idx(int n, const double* __restrict__ x, double* __restrict__ Y, long ld,
                           const int* __restrict__ jp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Y[(size_t)(*jp) * ld + i] = x[i];
}
// coefficients of step j to host-mapped slot j % 2, then j <- j + 1 (one block)
__global__ void k_export_step(const double* __restrict__ gs, int len, double* host_slots, int* jp) {
  const int j = *jp;
  double* dst = host_slots + (size_t)(j & 1) * len;
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = gs[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();
    *jp = j + 1;
  }
}

__global__ void k_multi_axpy(int n, int nvec, const double* __restrict__ V, long ld, const double* __restrict__ coef,
                             double* __restrict__ w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = w[i];
  for (int k = 0; k < nvec; ++k) acc -= coef[k] * V[(size_t)k * ld + i];
  w[i] = acc;
}
__global__ void k_combine(int n, int nvec, const double* __restrict__ V, long ld, const double* __restrict__ coef,
                          double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int k = 0; k < nvec; ++k) acc += coef[k] * V[(size_t)k * ld + i];
  y[i] = acc;
}
__global__ void k_normalize(int n, const double* w, const double* nrm2, double* v, double* h_slot) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double nr = sqrt(*nrm2);
  if (i < n) v[i] = (nr > 0.0) ? w[i] / nr : 0.0;
  if (i == 0 && h_slot) *h_slot = nr;
}
__global__ void k_cg_alpha(const double* rz, const double* pAp, double* alpha) { *alpha = *rz / *pAp; }
__global__ void k_cg_update_xr(int n, const double* alpha, const double* p, const double* Ap, double* x, double* r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = *alpha;
  x[i] += a * p[i];
  r[i] -= a * Ap[i];
}
__global__ void k_cg_update_p(int n, const double* rz_new, const double* rz_old, const double* z, double* p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double beta = *rz_new / *rz_old;
  p[i] = z[i] + beta * p[i];
}
__global__ void k_copy_scalar(const double* a, double* b) { *b = *a; }
__global__ void k_nonfinite(int n, const double* x, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicExch(&flags[FLAG_NONFINITE], 1);
}

}  // namespace

void launch_bsr_spmv(int nv, const int32_t* rp, const int32_t* col, const double* val, const double* x, double* y,
                     cudaStream_t s, const Mask& mk) {
  g_launches += 1;
  k_bsr_spmv_hw<double><<<nblk(16L * nv, 256), 256, 0, s>>>(nv, rp, col, val, x, y, nullptr, 0, mk);
}
void launch_bsr_spmv32(int nv, const int32_t* rp, const int32_t* col, const float* val, const double* x, double* y,
                       cudaStream_t s, const Mask& mk) {
  g_launches += 1;
  k_bsr_spmv_hw<float><<<nblk(16L * nv, 256), 256, 0, s>>>(nv, rp, col, val, x, y, nullptr, 0, mk);
}
void launch_bsr_spmv_ff(int nv, const int32_t* rp, const int32_t* col, const float* val, const float2* x2,
                        double* ybase, long yld, const int* jp, cudaStream_t s, const Mask& mk) {
  g_launches += 1;
  k_bsr_spmv_ff<<<nblk(16L * nv, 256), 256, 0, s>>>(nv, rp, col, val, x2, ybase, jp, yld, mk);
}
void launch_split(int n, const double* x, float2* x2, cudaStream_t s) {
  g_launches += 1;
  k_split<<<nblk(n, 256), 256, 0, s>>>(n, x, x2);
}
void launch_diag_inv(int nv, const int32_t* diag_slot, const double* val, const float* val32, double* dinv,
                     cudaStream_t s) {
  g_launches += 1;
  k_diag_inv<<<nblk(3L * nv, 256), 256, 0, s>>>(nv, diag_slot, val, val32, dinv);
}
// the product kernels at the scene's chunk length (entries per warp: 32 x 4, 8 or 16 per lane)
template <typename V, typename X, typename Y, typename Acc>
static void range_product(const SinvArgs& a, const V* val, const X* x, Y* y, cudaStream_t s, const Mask& mk) {
  const dim3 g(nblk(32L * a.nS, 256));
  if (a.chunk == 128)
    k_spmv_range_chunks<V, X, Y, Acc, 4><<<g, 256, 0, s>>>(a.nS, a.S_crow, a.S_cbeg, a.S_cend, a.S_c0, val, x, y, mk);
  else if (a.chunk == 512)
    k_spmv_range_chunks<V, X, Y, Acc, 16><<<g, 256, 0, s>>>(a.nS, a.S_crow, a.S_cbeg, a.S_cend, a.S_c0, val, x, y, mk);
  else
    k_spmv_range_chunks<V, X, Y, Acc, 8><<<g, 256, 0, s>>>(a.nS, a.S_crow, a.S_cbeg, a.S_cend, a.S_c0, val, x, y, mk);
}
template <typename V, typename X, typename Y, typename Acc>
static void transpose_product(const SinvArgs& a, const V* val, const X* w, Y* y, cudaStream_t s, const Mask& mk) {
  const dim3 g(nblk(32L * a.nSt, 256));
  if (a.chunk == 128)
    k_spmv_chunks<V, X, Y, Acc, 4><<<g, 256, 0, s>>>(a.nSt, a.St_crow, a.St_cbeg, a.St_cend, a.St_col, val, a.perm, w,
                                                     y, nullptr, 0, mk);
  else if (a.chunk == 512)
    k_spmv_chunks<V, X, Y, Acc, 16><<<g, 256, 0, s>>>(a.nSt, a.St_crow, a.St_cbeg, a.St_cend, a.St_col, val, a.perm, w,
                                                      y, nullptr, 0, mk);
  else
    k_spmv_chunks<V, X, Y, Acc, 8><<<g, 256, 0, s>>>(a.nSt, a.St_crow, a.St_cbeg, a.St_cend, a.St_col, val, a.perm, w,
                                                     y, nullptr, 0, mk);
}

void launch_sinv_half1(const SinvArgs& a, const double* x, double* w, cudaStream_t s, const Mask& mk) {
  g_launches += 2;
  k_to_position<double><<<nblk(3L * a.nv, 256), 256, 0, s>>>(a.nv, x, nullptr, 0, a.perm, a.xpos, mk);
  cudaMemsetAsync(w, 0, sizeof(double) * 3 * (size_t)a.nv, s);
  range_product<double, double, double, double>(a, a.S_val, a.xpos, w, s, mk);
}
void launch_sinv_half2(const SinvArgs& a, const double* w, double* y, cudaStream_t s, const Mask& mk) {
  g_launches += 1;
  cudaMemsetAsync(y, 0, sizeof(double) * 3 * (size_t)a.nv, s);
  transpose_product<double, double, double, double>(a, a.St_val, w, y, s, mk);
}
void launch_sinv_half1_32(const SinvArgs& a, const double* x, float* w32, cudaStream_t s, const Mask& mk) {
  g_launches += 2;
  k_to_position<float><<<nblk(3L * a.nv, 256), 256, 0, s>>>(a.nv, x, nullptr, 0, a.perm, a.xpos32, mk);
  cudaMemsetAsync(w32, 0, sizeof(float) * 3 * (size_t)a.nv, s);
  range_product<float, float, float, float>(a, a.S_val32, a.xpos32, w32, s, mk);
}
void launch_sinv_half2_32(const SinvArgs& a, const float* w32, double* y, cudaStream_t s, const Mask& mk) {
  g_launches += 1;
  cudaMemsetAsync(y, 0, sizeof(double) * 3 * (size_t)a.nv, s);
  transpose_product<float, float, double, float>(a, a.St_val32, w32, y, s, mk);
}
void launch_path_gather(int nc, const int32_t* cvertex, const int32_t* iperm, const SinvArgs& a, const double* w,
                        const float* w32, const double* frame, const double* cdata, int transpose, double* sc,
                        cudaStream_t s, const Mask& mk) {
  g_launches += 1;
  if (!nc) return;
  if (w32)
    k_path_gather<float, float><<<nblk(32L * nc, 256), 256, 0, s>>>(nc, cvertex, iperm, a.St_ptr, a.St_col,
                                                                    a.St_val32, w32, frame, cdata, transpose, sc, mk);
  else
    k_path_gather<double, double><<<nblk(32L * nc, 256), 256, 0, s>>>(nc, cvertex, iperm, a.St_ptr, a.St_col,
                                                                      a.St_val, w, frame, cdata, transpose, sc, mk);
}
void launch_path_scatter(int nc, const int32_t* cvertex, const int32_t* iperm, const SinvArgs& a, const double* frame,
                         const double* t, double coef, double* w, float* w32, cudaStream_t s, const Mask& mk) {
  g_launches += 1;
  if (!nc) return;
  if (w32)
    k_path_scatter<float, float><<<nblk(32L * nc, 256), 256, 0, s>>>(nc, cvertex, iperm, a.St_ptr, a.St_col,
                                                                     a.St_val32, frame, t, coef, w32, mk);
  else
    k_path_scatter<double, double><<<nblk(32L * nc, 256), 256, 0, s>>>(nc, cvertex, iperm, a.St_ptr, a.St_col,
                                                                       a.St_val, frame, t, coef, w, mk);
}

void launch_ainv(const SinvArgs& a, const double* x, double* w, double* y, cudaStream_t s) {
  launch_sinv_half1(a, x, w, s);
  launch_sinv_half2(a, w, y, s);
}
void launch_ainv32(const SinvArgs& a, const double* x, float* x32, float* w32, double* y, cudaStream_t s) {
  (void)x32;
  launch_sinv_half1_32(a, x, w32, s);
  launch_sinv_half2_32(a, w32, y, s);
}
void launch_contact_score(int nc, const int32_t* cvertex, const int32_t* iperm, const int64_t* St_ptr,
                          const double* St_val, const double* cdata, double h, double* score, cudaStream_t s) {
  g_launches += 1;
  if (nc) k_contact_score<<<nblk(32L * nc, 256), 256, 0, s>>>(nc, cvertex, iperm, St_ptr, St_val, cdata, h * h, score);
}
void launch_gather_contacts(int nk, const int32_t* idx, const int32_t* vertex, const double* frame,
                            const double* cdata, int32_t* ov, double* of, double* oc, cudaStream_t s) {
  g_launches += 1;
  if (nk) k_gather_contacts<<<nblk(nk, 128), 128, 0, s>>>(nk, idx, vertex, frame, cdata, ov, of, oc);
}
void launch_binding_capdata(int nb, const int32_t* vertex, const double* compliance, int off, int32_t* ov,
                            double* of, double* oc, cudaStream_t s) {
  g_launches += 1;
  if (nb) k_binding_capdata<<<nblk(nb, 128), 128, 0, s>>>(nb, vertex, compliance, off, ov, of, oc);
}
void launch_delassus(int nc, const int32_t* cvertex, const int32_t* iperm, const int64_t* St_ptr,
                     const int32_t* St_col, const double* St_val, double* Ds, cudaStream_t s) {
  g_launches += 1;
  k_delassus<<<nblk((long)nc * nc, 128), 128, 0, s>>>(nc, cvertex, iperm, St_ptr, St_col, St_val, Ds);
}
void launch_cap_form(int nc, const double* Ds, const double* frame, const double* cdata, double h, int transpose,
                     double* C, cudaStream_t s) {
  g_launches += 1;
  const long n = 3L * nc;
  k_cap_form<<<nblk(n * n, 256), 256, 0, s>>>(nc, Ds, frame, cdata, h * h, transpose, C);
}

__global__ void k_to_float_n(long n, const double* __restrict__ x, float* __restrict__ y) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
void launch_convert_f32(long n, const double* x, float* y, cudaStream_t s) {
  g_launches += 1;
  k_to_float_n<<<nblk(n, 256), 256, 0, s>>>(n, x, y);
}
void launch_gj_apply(int n, const double* B, const int32_t* piv, const double* y, double* ytmp, double* x,
                     cudaStream_t s, const int* act, int scene) {
  (void)ytmp;
  g_launches += 1;
  k_cap_apply<double><<<(n + 3) / 4, 256, sizeof(double) * (size_t)n, s>>>(n, B, piv, y, x, act, scene);
}
void launch_gj_apply32(int n, const float* B, const int32_t* piv, const double* y, double* ytmp, double* x,
                       cudaStream_t s, const int* act, int scene) {
  (void)ytmp;
  g_launches += 1;
  k_cap_apply<float><<<(n + 3) / 4, 256, sizeof(float) * (size_t)n, s>>>(n, B, piv, y, x, act, scene);
}
void launch_axpby(int n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
  g_launches += 1;
  k_axpby<<<nblk(n, 256), 256, 0, s>>>(n, a, x, b, y, out);
}
void launch_rhs(int n, const double* dq, const double* dv, double inv_h, double* b, cudaStream_t s) {
  g_launches += 1;
  k_rhs<<<nblk(n, 256), 256, 0, s>>>(n, dq, dv, inv_h, b);
}
void launch_mul(int n, const double* a, const double* b, double* y, cudaStream_t s) {
  g_launches += 1;
  k_mul<<<nblk(n, 256), 256, 0, s>>>(n, a, b, y);
}
void launch_multi_dot(int n, int nvec, const double* V, long ld, const double* w, double* partial, double* out,
                      cudaStream_t s) {
  // partial holds 64 * nvec doubles followed by nvec zero-initialised counters (see dot_scratch_doubles)
  g_launches += 1;
  int nb = nblk(n, 256);
  if (nb > 64) nb = 64;
  unsigned* cnt = reinterpret_cast<unsigned*>(partial + 64 * (size_t)kMaxDotVectors);
  k_multi_dot_fused<<<dim3(nb, nvec), 256, 0, s>>>(n, V, ld, w, partial, cnt, out);
}
void launch_multi_dot_idx(int n, int mmax, const double* V, long ld, const int* jp, bool self, double* partial,
                          double* out, cudaStream_t s) {
  g_launches += 1;
  int nb = nblk(n, 256);
  if (nb > 64) nb = 64;
  unsigned* cnt = reinterpret_cast<unsigned*>(partial + 64 * (size_t)kMaxDotVectors);
  k_multi_dot_idx<<<dim3(nb, self ? 1 : mmax + 1), 256, 0, s>>>(n, V, ld, jp, self ? 1 : 0, partial, cnt, out);
}
void launch_multi_axpy_idx(int n, const double* V, long ld, const int* jp, const double* coef, double* Vw,
                           cudaStream_t s) {
  g_launches += 1;
  k_multi_axpy_idx<<<nblk(n, 32), 256, 0, s>>>(n, V, ld, jp, coef, Vw);
}
void launch_normalize_idx(int n, double* V, long ld, const int* jp, const double* nrm2, double* h_slot, cudaStream_t s) {
  g_launches += 1;
  k_normalize_idx<<<nblk(n, 256), 256, 0, s>>>(n, V, ld, jp, nrm2, h_slot);
}
void launch_copy_idx(int n, const double* x, double* Y, long ld, const int* jp, cudaStream_t s) {
  g_launches += 1;
  k_copy_idx<<<nblk(n, 256), 256, 0, s>>>(n, x, Y, ld, jp);
}
void launch_export_step(const double* gs, int len, double* host_slots, int* jp, cudaStream_t s) {
  g_launches += 1;
  k_export_step<<<1, 256, 0, s>>>(gs, len, host_slots, jp);
}
void launch_bsr_spmv_idx(int nv, const int32_t* rp, const int32_t* col, const double* val, const float* val32,
                         const double* x, double* ybase, long yld, const int* jp, cudaStream_t s, const Mask& mk) {
  g_launches += 1;
  if (val32) k_bsr_spmv_hw<float><<<nblk(16L * nv, 256), 256, 0, s>>>(nv, rp, col, val32, x, ybase, jp, yld, mk);
  else k_bsr_spmv_hw<double><<<nblk(16L * nv, 256), 256, 0, s>>>(nv, rp, col, val, x, ybase, jp, yld, mk);
}
void launch_sinv_half1_idx(const SinvArgs& a, const double* xbase, long xld, const int* jp, double* w, float* w32,
                           cudaStream_t s, const Mask& mk) {
  g_launches += 2;
  if (w32) {
    k_to_position<float><<<nblk(3L * a.nv, 256), 256, 0, s>>>(a.nv, xbase, jp, xld, a.perm, a.xpos32, mk);
    cudaMemsetAsync(w32, 0, sizeof(float) * 3 * (size_t)a.nv, s);
    range_product<float, float, float, float>(a, a.S_val32, a.xpos32, w32, s, mk);
  } else {
    k_to_position<double><<<nblk(3L * a.nv, 256), 256, 0, s>>>(a.nv, xbase, jp, xld, a.perm, a.xpos, mk);
    cudaMemsetAsync(w, 0, sizeof(double) * 3 * (size_t)a.nv, s);
    range_product<double, double, double, double>(a, a.S_val, a.xpos, w, s, mk);
  }
}
void launch_multi_axpy(int n, int nvec, const double* V, long ld, const double* coef, double* w, cudaStream_t s) {
  g_launches += 1;
  k_multi_axpy<<<nblk(n, 256), 256, 0, s>>>(n, nvec, V, ld, coef, w);
}
void launch_combine(int n, int nvec, const double* V, long ld, const double* coef, double* y, cudaStream_t s) {
  g_launches += 1;
  k_combine<<<nblk(n, 256), 256, 0, s>>>(n, nvec, V, ld, coef, y);
}
void launch_normalize(int n, const double* w, const double* nrm2, double* v, double* h_slot, cudaStream_t s) {
  g_launches += 1;
  k_normalize<<<nblk(n, 256), 256, 0, s>>>(n, w, nrm2, v, h_slot);
}
void launch_cg_alpha(const double* rz, const double* pAp, double* alpha, cudaStream_t s) {
  g_launches += 1;
  k_cg_alpha<<<1, 1, 0, s>>>(rz, pAp, alpha);
}
void launch_cg_update_xr(int n, const double* alpha, const double* p, const double* Ap, double* x, double* r,
                         cudaStream_t s) {
  g_launches += 1;
  k_cg_update_xr<<<nblk(n, 256), 256, 0, s>>>(n, alpha, p, Ap, x, r);
}
void launch_cg_update_p(int n, const double* rz_new, const double* rz_old, const double* z, double* p,
                        cudaStream_t s) {
  g_launches += 1;
  k_cg_update_p<<<nblk(n, 256), 256, 0, s>>>(n, rz_new, rz_old, z, p);
}
void launch_copy_scalar(const double* src, double* dst, cudaStream_t s) {
  g_launches += 1; k_copy_scalar<<<1, 1, 0, s>>>(src, dst); }
void launch_nonfinite_check(int n, const double* x, int* flags, cudaStream_t s) {
  g_launches += 1;
  k_nonfinite<<<nblk(n, 256), 256, 0, s>>>(n, x, flags);
}

}  // namespace ncpadj
