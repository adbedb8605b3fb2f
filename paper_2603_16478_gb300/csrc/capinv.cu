// Capacitance blocks of the Woodbury preconditioner (Sec. 4.4) as tables: the Delassus blocks and
// capacitances of every block in two launches, the inverses of the small blocks one CTA each in one
// launch, and the one-launch apply of every block's inverse.  (The large blocks are inverted by the
// pivoted Gauss-Jordan of gj.cu or the tensor-core blocked Gauss-Jordan of bgj.cu.)
#include <stdint.h>

#include "kernels.cuh"

namespace ncpadj {
namespace {

// In-place inverses of many small blocks in one launch, one CTA per block: block ids[bx] of the table
// meta (element offset [nb], row offset [nb], dimension [nb]) is loaded into shared memory (row
// stride n + 1), inverted by Gauss-Jordan with row pivoting, written back as the
// inverse itself, and its pivot entries set to the identity (the apply kernels take it as it is).
// A zero pivot raises FLAG_SINGULAR and leaves the block as it was.
template <typename T>
__global__ void __launch_bounds__(256) k_small_inverse(int nsmall, const int32_t* __restrict__ ids, int nb,
                                                       const int64_t* __restrict__ meta, T* __restrict__ Bs,
                                                       int32_t* __restrict__ piv_out, int* flags) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int k = ids[blockIdx.x];
  const int64_t moff = meta[k], o = meta[nb + k];
  const int n = (int)meta[2 * nb + k], ld = n + 1;
  T* S = reinterpret_cast<T*>(smraw);
  T* col = S + (size_t)n * ld;
  T* row = col + n;
  int* piv = reinterpret_cast<int*>(row + n);
  __shared__ int bad;
  T* M = Bs + moff;
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += blockDim.x) S[(e / n) * ld + e % n] = M[e];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (tid < 32) {
      T best = T(-1);
      int arg = c;
      for (int i = c + tid; i < n; i += 32) {
        const T v = fabs(S[i * ld + c]);
        if (v > best) {
          best = v;
          arg = i;
        }
      }
      for (int w = 16; w > 0; w >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, w);
        const int oa = __shfl_down_sync(0xffffffffu, arg, w);
        if (ob > best || (ob == best && oa < arg)) {
          best = ob;
          arg = oa;
        }
      }
      if (tid == 0) {
        piv[c] = arg;
        if (!(best > T(0))) bad = 1;
      }
    }
    __syncthreads();
    if (bad) break;
    const int p = piv[c];
    if (p != c)
      for (int j = tid; j < n; j += blockDim.x) {
        const T t = S[c * ld + j];
        S[c * ld + j] = S[p * ld + j];
        S[p * ld + j] = t;
      }
    __syncthreads();
    for (int j = tid; j < n; j += blockDim.x) {
      col[j] = S[j * ld + c];
      row[j] = S[c * ld + j];
    }
    __syncthreads();
    const T inv = T(1) / row[c];
    for (int e = tid; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e % n;
      if (i == c) S[i * ld + j] = (j == c) ? inv : row[j] * inv;
      else S[i * ld + j] = (j == c) ? -col[i] * inv : S[i * ld + j] - col[i] * row[j] * inv;
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicExch(&flags[FLAG_SINGULAR], 1);
    return;
  }
  for (int c = n - 1; c >= 0; --c) {
    const int p = piv[c];
    if (p != c)
      for (int i = tid; i < n; i += blockDim.x) {
        const T t = S[i * ld + c];
        S[i * ld + c] = S[i * ld + p];
        S[i * ld + p] = t;
      }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += blockDim.x) M[e] = S[(e / n) * ld + e % n];
  for (int j = tid; j < n; j += blockDim.x) piv_out[o + j] = j;
}

// x_k = B_k y_k for every capacitance block k at once (one launch instead of one per block): meta
// holds [nb] element offsets of the blocks' inverses, [nb] offsets of their rows in y and x (3 c0),
// [nb] dimensions and [nb] scenes.  Block (bx, k) computes rows 4 bx .. 4 bx + 3 of block k from y
// staged in shared memory with the block's pivots, two warps per row; a block whose scene is idle
// (act) or that has fewer rows does nothing.
__device__ __forceinline__ float lane_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double lane_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_cap_apply_all(int nb, const int64_t* __restrict__ meta,
                                                       const T* __restrict__ Bs, const int32_t* __restrict__ piv,
                                                       const double* __restrict__ y, double* __restrict__ x,
                                                       const int* __restrict__ act, int accumulate) {
  const int k = blockIdx.y;
  const int64_t moff = meta[k], o = meta[nb + k];
  const int n = (int)meta[2 * nb + k], scene = (int)meta[3 * nb + k];
  if (act && !act[scene]) return;
  if ((int)blockIdx.x * 4 >= n) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* ys = reinterpret_cast<T*>(smraw);
  __shared__ T part[4][2];
  const int32_t* pv = piv + o;
  for (int j = threadIdx.x; j < n; j += blockDim.x) ys[j] = (T)y[o + pv[j]];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rloc = warp >> 1, half = warp & 1;
  const int r = blockIdx.x * 4 + rloc;
  T acc = 0;
  if (r < n) {
    const T* row = Bs + moff + (size_t)pv[r] * n;
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
  acc = lane_sum(acc);
  if (lane == 0) part[rloc][half] = acc;
  __syncthreads();
  if (threadIdx.x < 4) {
    const int rr = blockIdx.x * 4 + threadIdx.x;
    if (rr < n) {
      const double v = (double)(part[threadIdx.x][0] + part[threadIdx.x][1]);
      x[o + rr] = accumulate ? x[o + rr] + v : v;
    }
  }
}

// r_k = y_k - C_k x_k in FP64 for every capacitance block k (C_k the capacitance itself, row-major at
// C + meta[k], unpermuted; x_k in natural order): the residual of one step of iterative refinement.
// Layout as k_cap_apply_all: block (bx, k) takes rows 4 bx .. 4 bx + 3, two warps per row, x_k staged
// in shared memory.
__global__ void __launch_bounds__(256) k_cap_resid_all(int nb, const int64_t* __restrict__ meta,
                                                       const double* __restrict__ C, const double* __restrict__ y,
                                                       const double* __restrict__ x, double* __restrict__ r,
                                                       const int* __restrict__ act) {
  const int k = blockIdx.y;
  const int64_t moff = meta[k], o = meta[nb + k];
  const int n = (int)meta[2 * nb + k], scene = (int)meta[3 * nb + k];
  if (act && !act[scene]) return;
  if ((int)blockIdx.x * 4 >= n) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* xs = reinterpret_cast<double*>(smraw);
  __shared__ double part[4][2];
  for (int j = threadIdx.x; j < n; j += blockDim.x) xs[j] = x[o + j];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rloc = warp >> 1, half = warp & 1;
  const int row_i = blockIdx.x * 4 + rloc;
  double acc = 0;
  if (row_i < n) {
    const double* row = C + moff + (size_t)row_i * n;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int j = half * 32 + lane;
    for (; j + 192 < n; j += 256) {
      a0 += row[j] * xs[j];
      a1 += row[j + 64] * xs[j + 64];
      a2 += row[j + 128] * xs[j + 128];
      a3 += row[j + 192] * xs[j + 192];
    }
    for (; j < n; j += 64) a0 += row[j] * xs[j];
    acc = (a0 + a1) + (a2 + a3);
  }
  acc = lane_sum(acc);
  if (lane == 0) part[rloc][half] = acc;
  __syncthreads();
  if (threadIdx.x < 4) {
    const int rr = blockIdx.x * 4 + threadIdx.x;
    if (rr < n) r[o + rr] = y[o + rr] - (part[threadIdx.x][0] + part[threadIdx.x][1]);
  }
}

// The capacitance of every block of the table in two launches (instead of two per block).  meta
// rows: element offset of C_k, 3 c0_k, n_k = 3 m_k, scene, offset of D_k.
// D_k[a][b] = sum_i S[i][p_a] S[i][p_b]: rows p_a, p_b of S^T are the elimination-tree paths of the
// contacts' positions, which share exactly the common suffix from their lowest common ancestor.
__global__ void k_delassus_all(int nb, const int64_t* __restrict__ meta, const int32_t* __restrict__ cvertex,
                               const int32_t* __restrict__ iperm, const int64_t* __restrict__ ptr,
                               const int32_t* __restrict__ col, const double* __restrict__ val, double* __restrict__ Ds) {
  const int k = blockIdx.y;
  const int c0 = (int)(meta[nb + k] / 3), m = (int)(meta[2 * nb + k] / 3);
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)m * m) return;
  const int a = (int)(idx / m), b = (int)(idx - (long)a * m);
  const int ia = iperm[cvertex[c0 + a]], ib = iperm[cvertex[c0 + b]];
  int64_t pa = ptr[ia + 1] - 1, pb = ptr[ib + 1] - 1;
  const int64_t ea = ptr[ia], eb = ptr[ib];
  double acc = 0.0;
  while (pa >= ea && pb >= eb && col[pa] == col[pb]) {
    acc += val[pa] * val[pb];
    --pa;
    --pb;
  }
  Ds[meta[4 * nb + k] + idx] = acc;
}

// C_k[3a+r][3b+s] = delta + h^2 D_k[a][b] sum_l K'_a[r][l] (F_a F_b^T)[l][s], K' = K^T (adjoint) or K;
// written in FP64 and, when C32 is given, rounded to FP32 beside it
__global__ void k_cap_form_all(int nb, const int64_t* __restrict__ meta, const double* __restrict__ Ds,
                               const double* __restrict__ frame, const double* __restrict__ cdata, double h2,
                               int transpose, double* __restrict__ C, float* __restrict__ C32) {
  const int k = blockIdx.y;
  const int c0 = (int)(meta[nb + k] / 3);
  const long n = meta[2 * nb + k], m = n / 3;
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int R = (int)(idx / n), Cc = (int)(idx - (long)R * n);
  const int a = R / 3, r = R - 3 * a, b = Cc / 3, sdx = Cc - 3 * b;
  const double* Fa = frame + 9 * (size_t)(c0 + a);
  const double* Fb = frame + 9 * (size_t)(c0 + b);
  const double* Ka = cdata + 12 * (size_t)(c0 + a);
  double acc = 0.0;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const double ff = Fa[3 * l] * Fb[3 * sdx] + Fa[3 * l + 1] * Fb[3 * sdx + 1] + Fa[3 * l + 2] * Fb[3 * sdx + 2];
    acc += (transpose ? Ka[3 * l + r] : Ka[3 * r + l]) * ff;
  }
  const double v = (R == Cc ? 1.0 : 0.0) + h2 * Ds[meta[4 * nb + k] + (size_t)a * m + b] * acc;
  C[meta[k] + idx] = v;
  if (C32) C32[meta[k] + idx] = (float)v;
}

__global__ void k_fill(long n, double v, double* x) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

}  // namespace

void launch_fill(long n, double v, double* x, cudaStream_t s) {
  if (n <= 0) return;
  g_launches += 1;
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, v, x);
}

void launch_cap_form_all(int nb, int mmax, const int64_t* meta, const int32_t* cvertex, const int32_t* iperm,
                         const int64_t* St_ptr, const int32_t* St_col, const double* St_val, double* Ds,
                         const double* frame, const double* cdata, double h, int transpose, double* C, float* C32,
                         cudaStream_t s) {
  if (nb <= 0 || mmax <= 0) return;
  g_launches += 2;
  const long mm = (long)mmax * mmax, nn = 9L * mm;
  k_delassus_all<<<dim3((unsigned)((mm + 127) / 128), nb), 128, 0, s>>>(nb, meta, cvertex, iperm, St_ptr, St_col,
                                                                         St_val, Ds);
  k_cap_form_all<<<dim3((unsigned)((nn + 255) / 256), nb), 256, 0, s>>>(nb, meta, Ds, frame, cdata, h * h, transpose,
                                                                         C, C32);
}

void launch_cap_apply_all(int nb, int nmax, const int64_t* meta, const float* B32, const double* B64,
                          const int32_t* piv, const double* y, double* x, const int* act, cudaStream_t s,
                          bool accumulate) {
  if (nb <= 0 || nmax <= 0) return;
  g_launches += 1;
  const dim3 grid((nmax + 3) / 4, nb);
  if (B32)
    k_cap_apply_all<float><<<grid, 256, sizeof(float) * (size_t)nmax, s>>>(nb, meta, B32, piv, y, x, act, accumulate);
  else
    k_cap_apply_all<double><<<grid, 256, sizeof(double) * (size_t)nmax, s>>>(nb, meta, B64, piv, y, x, act, accumulate);
}

void launch_cap_resid_all(int nb, int nmax, const int64_t* meta, const double* C, const double* y, const double* x,
                          double* r, const int* act, cudaStream_t s) {
  if (nb <= 0 || nmax <= 0) return;
  g_launches += 1;
  const size_t sm = sizeof(double) * (size_t)nmax;
  if (sm > 48 * 1024)  // per device: set on every call that needs it
    cudaFuncSetAttribute(k_cap_resid_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_cap_resid_all<<<dim3((nmax + 3) / 4, nb), 256, sm, s>>>(nb, meta, C, y, x, r, act);
}

int small_inverse_max(bool fp32) { return fp32 ? 192 : 128; }

static size_t small_inverse_smem(int n, size_t es) { return es * ((size_t)n * (n + 1) + 2 * (size_t)n) + 4 * (size_t)n; }

void launch_small_inverse(int nsmall, const int32_t* ids, int nb, const int64_t* meta, int nmax, float* B32,
                          double* B64, int32_t* piv, int* flags, cudaStream_t s) {
  if (nsmall <= 0) return;
  g_launches += 1;
  if (B32) {
    const size_t sm = small_inverse_smem(nmax, sizeof(float));
    cudaFuncSetAttribute(k_small_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_small_inverse<float><<<nsmall, 256, sm, s>>>(nsmall, ids, nb, meta, B32, piv, flags);
  } else {
    const size_t sm = small_inverse_smem(nmax, sizeof(double));
    cudaFuncSetAttribute(k_small_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_small_inverse<double><<<nsmall, 256, sm, s>>>(nsmall, ids, nb, meta, B64, piv, flags);
  }
}

}  // namespace ncpadj
