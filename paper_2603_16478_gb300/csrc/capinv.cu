// Inverse of a dense FP32 matrix by Schur-complement recursion with tensor-core GEMMs: the
// capacitance inverse of the Woodbury preconditioner (Sec. 4.4) when it is taken in FP32.
//
// For M = [[A, B], [C, D]] (A the leading n1 x n1 block):
//   A <- A^{-1};  X = A^{-1} B;  Y = C A^{-1};  D <- S = D - C X;  D <- S^{-1};
//   B <- -X S^{-1};  A <- A^{-1} - B Y;  C <- -S^{-1} Y,
// which leaves M^{-1} in place.  The six products per level run on tcgen05 (tc.cu, 3xTF32); blocks of
// at most kLeaf rows are inverted by one CTA in shared memory by Gauss-Jordan elimination with row
// pivoting inside the block (the recursion itself does not pivot, so a leading block must be
// invertible: the capacitance I + h^2 K^T D is, in the cases the tests cover).  Every launch goes to
// the caller's stream; nothing waits on the host.
#include <stdint.h>

#include "kernels.cuh"

namespace ncpadj {
namespace {

constexpr int kLeaf = 64;        // rows of a block inverted in shared memory
constexpr int kLeafThreads = 256;

// In-place inverse of the b x b block at M (row stride ld), b <= kLeaf: Gauss-Jordan with the
// pivot of largest magnitude in the column (rows k..b-1), the row interchanges undone on the columns
// at the end.  A zero pivot raises FLAG_SINGULAR (the block is left as it is).
__global__ void __launch_bounds__(kLeafThreads) k_leaf_inverse(int b, float* M, long ld, int* flags) {
  __shared__ float S[kLeaf][kLeaf + 1];
  __shared__ float col[kLeaf], row[kLeaf];
  __shared__ int piv[kLeaf];
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += kLeafThreads) S[e / b][e % b] = M[(long)(e / b) * ld + e % b];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < b; ++k) {
    if (tid < 32) {  // pivot search by the first warp
      float best = -1.0f;
      int arg = k;
      for (int i = k + tid; i < b; i += 32) {
        const float v = fabsf(S[i][k]);
        if (v > best) {
          best = v;
          arg = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oa = __shfl_down_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) {
          best = ob;
          arg = oa;
        }
      }
      if (tid == 0) {
        piv[k] = arg;
        if (!(best > 0.0f)) bad = 1;
      }
    }
    __syncthreads();
    if (bad) break;
    const int p = piv[k];
    if (p != k)
      for (int j = tid; j < b; j += kLeafThreads) {
        const float t = S[k][j];
        S[k][j] = S[p][j];
        S[p][j] = t;
      }
    __syncthreads();
    for (int j = tid; j < b; j += kLeafThreads) {
      col[j] = S[j][k];
      row[j] = S[k][j];
    }
    __syncthreads();
    const float inv = 1.0f / row[k];
    for (int e = tid; e < b * b; e += kLeafThreads) {
      const int i = e / b, j = e % b;
      if (i == k) S[i][j] = (j == k) ? inv : row[j] * inv;
      else S[i][j] = (j == k) ? -col[i] * inv : S[i][j] - col[i] * row[j] * inv;
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicExch(&flags[FLAG_SINGULAR], 1);
    return;
  }
  for (int k = b - 1; k >= 0; --k) {  // undo the row interchanges on the columns
    const int p = piv[k];
    if (p != k)
      for (int i = tid; i < b; i += kLeafThreads) {
        const float t = S[i][k];
        S[i][k] = S[i][p];
        S[i][p] = t;
      }
    __syncthreads();
  }
  for (int e = tid; e < b * b; e += kLeafThreads) M[(long)(e / b) * ld + e % b] = S[e / b][e % b];
}

__global__ void k_iota(int n, int32_t* p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

void gemm(int M, int N, int K, float alpha, const float* A, long lda, const float* B, long ldb, float beta, float* C,
          long ldc, int* flags, cudaStream_t s) {
  launch_tc_gemm(GemmArgs{M, N, K, alpha, beta, A, lda, B, ldb, C, ldc, 1, flags}, s);
}

// M (n x n, row stride ld) <- M^{-1}; scratch holds rec_inverse_scratch(n) floats
void rec_inverse(int n, float* M, long ld, float* scratch, int* flags, cudaStream_t s) {
  if (n <= kLeaf) {
    g_launches += 1;
    k_leaf_inverse<<<1, kLeafThreads, 0, s>>>(n, M, ld, flags);
    return;
  }
  const int n1 = kLeaf * ((n / kLeaf + 1) / 2), n2 = n - n1;
  float* A = M;
  float* B = M + n1;
  float* C = M + (long)n1 * ld;
  float* D = C + n1;
  float* X = scratch;                  // n1 x n2
  float* Y = scratch + (long)n1 * n2;  // n2 x n1
  rec_inverse(n1, A, ld, scratch, flags, s);
  gemm(n1, n2, n1, 1.0f, A, ld, B, ld, 0.0f, X, n2, flags, s);    // X = A^-1 B
  gemm(n2, n1, n1, 1.0f, C, ld, A, ld, 0.0f, Y, n1, flags, s);    // Y = C A^-1
  gemm(n2, n2, n1, -1.0f, C, ld, X, n2, 1.0f, D, ld, flags, s);   // D = D - C X
  rec_inverse(n2, D, ld, scratch + 2 * (long)n1 * n2, flags, s);  // D = S^-1
  gemm(n1, n2, n2, -1.0f, X, n2, D, ld, 0.0f, B, ld, flags, s);   // B = -X S^-1
  gemm(n1, n1, n2, -1.0f, B, ld, Y, n1, 1.0f, A, ld, flags, s);   // A = A^-1 - B Y
  gemm(n2, n1, n2, -1.0f, D, ld, Y, n1, 0.0f, C, ld, flags, s);   // C = -S^-1 Y
}

}  // namespace

size_t rec_inverse_scratch(int n) { return (size_t)n * n + 64; }

void launch_rec_inverse(int n, float* M, long ld, float* scratch, int32_t* piv, int* flags, cudaStream_t s) {
  if (n <= 0) return;
  rec_inverse(n, M, ld, scratch, flags, s);
  if (piv) {  // the result is the inverse itself: the identity permutation for the Gauss-Jordan apply
    g_launches += 1;
    k_iota<<<(n + 255) / 256, 256, 0, s>>>(n, piv);
  }
}

}  // namespace ncpadj
