// Dense FP32 GEMM on the fifth-generation tensor cores (tcgen05, kind::tf32), the dense product of
// the capacitance inverse (Sec. 4.4, Woodbury preconditioner; bgj.cu runs the same MMA inside its
// persistent kernel), exposed on its own through ncpadj_dense_gemm.
//
//   C = alpha A B + beta C,   A [M][K], B [K][N], C [M][N] row-major FP32 with leading dimensions.
//
// One CTA of 128 threads computes a 128 x 128 tile of C.  Per K-slab of 32 the threads stage A's rows
// and B's columns into shared memory in the canonical no-swizzle K-major layout of the MMA (core
// matrices of 8 rows x 16 bytes; the next core matrix along K 128 bytes on, the next 8 rows 256 bytes
// on), fence the generic-proxy stores for the async proxy, and one elected thread issues four
// tcgen05.mma (M = 128, N = 128, K = 8 each) into a 128-column TMEM accumulator and commits them to an
// mbarrier.  Every wait on the mbarrier has an iteration limit: past it the kernel raises
// FLAG_TIMEOUT, skips the epilogue, frees its TMEM and returns.  The epilogue reads the accumulator
// with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e. rows 32w.. of the tile).
//
// split = 1 (3xTF32): each operand x is split into its TF32 rounding h = rna(x) and t = rna(x - h);
// h_A h_B + h_A t_B + t_A h_B, accumulated in FP32, recovers about FP32 accuracy (the dropped t_A t_B
// is ~2^-22 of the product).  split = 0 uses h only (TF32 accuracy).
#include <stdint.h>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace ncpadj {
namespace {

using namespace tc5;

constexpr int TM = 128, TN = 128, TK = 32;
constexpr int SLAB = kSlabBytes;      // one K = 8 slab of a 128-row operand tile (bytes)
constexpr int OPB = (TK / 8) * SLAB;  // a 128 x 32 operand tile (bytes)
constexpr int TMEM_COLS = 128;        // FP32 accumulator columns (= TN)
constexpr uint32_t kIdesc = idesc_tf32(TN);

__global__ void __launch_bounds__(128) k_tc_gemm(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned operand area: A_h, B_h (and A_t, B_t when split)
  unsigned char* sm = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
  unsigned char* sA = sm;
  unsigned char* sB = sm + OPB;
  unsigned char* sAt = sm + 2 * OPB;
  unsigned char* sBt = sm + 3 * OPB;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  if (tid == 0) {
    mbar_init(smem_addr(&mbar), 1);
    failed = 0;
  }
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const int nk = (g.K + TK - 1) / TK;
  uint32_t phase = 0;
  for (int kt = 0; kt < nk; ++kt) {
    const int k0 = kt * TK;
    // stage A rows m0.. and B columns n0.. of this K-slab (zero outside the matrices)
    for (int i = tid; i < TM * TK; i += 128) {
      const int r = i / TK, k = i % TK;
      const float a = (m0 + r < g.M && k0 + k < g.K) ? g.A[(long)(m0 + r) * g.lda + k0 + k] : 0.0f;
      const float ah = tf32_rna(a);
      *reinterpret_cast<float*>(sA + tile_off(r, k)) = ah;
      if (g.split) *reinterpret_cast<float*>(sAt + tile_off(r, k)) = tf32_rna(a - ah);
    }
    for (int i = tid; i < TN * TK; i += 128) {
      const int n = i % TN, k = i / TN;
      const float b = (n0 + n < g.N && k0 + k < g.K) ? g.B[(long)(k0 + k) * g.ldb + n0 + n] : 0.0f;
      const float bh = tf32_rna(b);
      *reinterpret_cast<float*>(sB + tile_off(n, k)) = bh;
      if (g.split) *reinterpret_cast<float*>(sBt + tile_off(n, k)) = tf32_rna(b - bh);
    }
    fence_smem_async();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      for (int s = 0; s < TK / 8; ++s) {
        const uint32_t acc = (kt > 0 || s > 0) ? 1u : 0u;
        const uint64_t ah = sdesc(smem_addr(sA + s * SLAB)), bh = sdesc(smem_addr(sB + s * SLAB));
        mma_tf32(tmem, ah, bh, kIdesc, acc);
        if (g.split) {
          mma_tf32(tmem, ah, sdesc(smem_addr(sBt + s * SLAB)), kIdesc, 1u);
          mma_tf32(tmem, sdesc(smem_addr(sAt + s * SLAB)), bh, kIdesc, 1u);
        }
      }
      mma_commit(smem_addr(&mbar));
    }
    // every thread waits for the MMAs (they read the shared tiles the next slab overwrites)
    if (!mbar_wait(smem_addr(&mbar), phase)) failed = 1;
    phase ^= 1u;
    __syncthreads();
    if (failed) break;
  }
  fence_after_sync();
  if (failed) {
    if (tid == 0) {
      atomicExch(&g.flags[FLAG_TIMEOUT], 1);
      mbar_wait(smem_addr(&mbar), phase ^ 1u);  // the MMAs in flight, once more (bounded), before the free
    }
  } else {
    const int r = warp * 32 + (tid & 31);  // TMEM lane = row of the tile
    for (int c = 0; c < TN; c += 8) {
      uint32_t v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      if (m0 + r < g.M) {
        float* crow = g.C + (long)(m0 + r) * g.ldc + n0 + c;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (n0 + c + j < g.N) {
            const float x = g.alpha * __uint_as_float(v[j]);
            crow[j] = (g.beta == 0.0f) ? x : x + g.beta * crow[j];
          }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

size_t tc_gemm_smem(int split) { return (size_t)(split ? 4 : 2) * OPB + 1024; }

void launch_tc_gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return;
  g_launches += 1;
  const size_t smem = tc_gemm_smem(g.split);
  static thread_local bool attr_set[2] = {false, false};
  if (!attr_set[g.split ? 1 : 0]) {
    cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_gemm_smem(1));
    attr_set[g.split ? 1 : 0] = true;
  }
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM);
  k_tc_gemm<<<grid, 128, smem, s>>>(g);
}

}  // namespace ncpadj
