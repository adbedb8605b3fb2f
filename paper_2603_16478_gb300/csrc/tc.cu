// Dense FP32 GEMM on the fifth-generation tensor cores (tcgen05, kind::tf32): the building block of
// the capacitance inverse's Schur-complement recursion (Sec. 4.4, Woodbury preconditioner).
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

namespace ncpadj {
namespace {

constexpr int TM = 128, TN = 128, TK = 32;
constexpr int SLAB = 128 * 8 * 4;       // one K = 8 slab of a 128-row operand tile (bytes)
constexpr int OPB = (TK / 8) * SLAB;    // a 128 x 32 operand tile (bytes)
constexpr int TMEM_COLS = 128;          // FP32 accumulator columns (= TN)
constexpr long kWaitLimit = 1L << 22;   // mbarrier polls before giving up

// instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle, K-major: start address, leading byte offset (next core
// matrix along K) 128, stride byte offset (next 8 rows) 256, descriptor version 1 (bits 46-47)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// byte offset of element (r, k) of a 128 x 32 K-major operand tile
__device__ __forceinline__ int tile_off(int r, int k) {
  return (k >> 3) * SLAB + (r >> 3) * 256 + ((k >> 2) & 1) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    failed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
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
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int s = 0; s < TK / 8; ++s) {
        const uint32_t acc = (kt > 0 || s > 0) ? 1u : 0u;
        const uint64_t ah = sdesc(smem_addr(sA + s * SLAB)), bh = sdesc(smem_addr(sB + s * SLAB));
        mma_tf32(tmem, ah, bh, acc);
        if (g.split) {
          mma_tf32(tmem, ah, sdesc(smem_addr(sBt + s * SLAB)), 1u);
          mma_tf32(tmem, sdesc(smem_addr(sAt + s * SLAB)), bh, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&mbar))
                   : "memory");
    }
    // every thread waits for the MMAs (they read the shared tiles the next slab overwrites)
    if (!mbar_wait(smem_addr(&mbar), phase)) failed = 1;
    phase ^= 1u;
    __syncthreads();
    if (failed) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (failed) {
    if (tid == 0) {
      atomicExch(&g.flags[FLAG_TIMEOUT], 1);
      mbar_wait(smem_addr(&mbar), phase ^ 1u);  // the MMAs in flight, once more (bounded), before the free
    }
  } else {
    const int r = warp * 32 + (tid & 31);  // TMEM lane = row of the tile
    for (int c = 0; c < TN; c += 8) {
      uint32_t v[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
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
