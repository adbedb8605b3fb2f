// Dense FP32 inverse of a capacitance matrix C = I + h^2 K'^T D (Woodbury preconditioner, Sec. 4.4)
// by blocked Gauss-Jordan elimination in ONE persistent cooperative launch, with the rank-64 updates
// on the tensor cores (tcgen05, kind::tf32, 3xTF32 split: about FP32 accuracy).
//
// Block step k eliminates the 64 columns K = [64k, 64k + 64) at once.  With D_k = M[K][K] and its
// inverse D_k^{-1} (pivoting among the block's own rows),
//   Lhat = M[:, K] with D_k - I in the rows K,        (n x 64)
//   R    = D_k^{-1} M[K, :] with D_k^{-1} in the columns K,   (64 x n)
//   M   <- Cold - Lhat R,  Cold = M except Cold[:, K] = E (the identity's columns K),
// which is the in-place Gauss-Jordan sweep of the whole block: after the last step M holds C^{-1}.
// Pivoting stays inside the 64 x 64 diagonal blocks, after the rows are equilibrated by powers of
// two (the capacitance's rows carry the contact stiffnesses K, which span many decades); a zero
// pivot raises FLAG_SINGULAR.
//
// Work per step, between two bounded grid barriers:
//   P2 (all CTAs but the last): Lhat and R^T, each split into TF32 head and tail, written in the
//      MMA's no-swizzle K-major tile layout (one 32 KB operand tile per 128 rows), so the tile
//      owners copy them straight into shared memory.  The last CTA meanwhile forms the next
//      diagonal block D_{k+1} = M[K',K'] - M[K',K] D_k^{-1} M[K,K'] from the same values (SIMT).
//   P3 (all CTAs but the last): each owned 128 x 128 tile of M gets Cold - Lhat_I R_J by 8 K-steps
//      of 3 MMAs into a TMEM accumulator, read back with tcgen05.ld, staged through shared memory
//      and applied to M row by row; the last CTA meanwhile inverts D_{k+1} (look-ahead), so the
//      critical path per step is P2, one 64 x 64 inverse and two barriers.
// Every wait (grid barriers, the MMA mbarrier) is bounded: past its limit the kernel raises
// FLAG_TIMEOUT and the abort word, every CTA leaves at its next barrier, and TMEM is freed.
#include <stdint.h>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace ncpadj {
namespace {

using namespace tc5;

constexpr int BB = 64;                     // columns eliminated per step
constexpr int BT = 128;                    // output tile (M = N of the MMA)
constexpr int kThreads = 256;
constexpr int kOpBytes = BT * BB * 4;      // one operand tile: 128 rows x 64 K, FP32 (32 KB)
constexpr int kOpFloats = kOpBytes / 4;
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kIdesc = idesc_tf32(BT);
constexpr long kBarrierLimit = 1L << 21;   // polls of a grid barrier (each >= 64 ns of sleep + an L2 load)

struct BgjArgs {
  int n;
  float* M;
  long ld;
  float *Lh, *Lt, *Rh, *Rt;  // [tiles][kOpFloats] operand tiles (TF32 head, tail) of Lhat and R^T
  float* Dd;                 // [2][64][64] the diagonal blocks as inverted (step parity)
  float* Dinv;               // [64][64] the current one's inverse
  float* rscale;             // [n] power-of-two row scales (equilibration)
  unsigned* sync;            // [0] arrivals, [1] generation, [2] abort
  int* flags;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch with a bounded wait.  False once any CTA has raised the
// abort word (its own wait ran out, a zero pivot, an MMA that never completed): the caller stops.
__device__ bool grid_barrier(unsigned* sync, unsigned& gen, int* flags) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned target = gen + 1;
    int good = 1;
    if (atomicAdd(&sync[0], 1u) == gridDim.x - 1) {
      atomicExch(&sync[0], 0u);
      __threadfence();
      st_release_u32(&sync[1], target);
    } else {
      long it = 0;
      while (ld_acquire_u32(&sync[1]) != target) {
        if (ld_acquire_u32(&sync[2])) {
          good = 0;
          break;
        }
        if (++it > kBarrierLimit) {
          atomicExch(&sync[2], 1u);
          atomicExch(&flags[FLAG_TIMEOUT], 1);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (good && ld_acquire_u32(&sync[2])) good = 0;
    gen = target;
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// 16-byte asynchronous global -> shared copy through L2 only (data written by other CTAs in this
// launch must not come from a stale L1 line)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void raise_abort(unsigned* sync) {
  __threadfence();
  atomicExch(&sync[2], 1u);
}

// float index of element (i, c) of an n x 64 operand stored as 128-row tiles in the MMA layout
__device__ __forceinline__ long op_index(int i, int c) {
  return (long)(i >> 7) * kOpFloats + (tile_off(i & 127, c) >> 2);
}

__device__ __forceinline__ void put_split(float* H, float* T, long idx, float v) {
  const float h = tf32_rna(v);
  H[idx] = h;
  T[idx] = tf32_rna(v - h);
}

// Inverse of the 64 x 64 block Ds (shared, row stride 65) by Gauss-Jordan elimination in place,
// without row interchanges: the pivot of column k is the row of largest magnitude among the rows not
// yet used.  Thread t keeps row t / 4, columns 16 (t % 4) .. + 15 in registers, so a column's 64
// values sit one per thread: the pivot search is a warp max (redux) of 32-bit keys and one exchange
// of eight warp candidates; the pivot row passes through shared memory, the column value within the
// row's four lanes by shuffle (two barriers per column).  With pivot rows p_k the result S
// satisfies C^{-1}[k][p_j] = S[p_k][j], which is how the inverse is written to Dinv.  Returns false
// (Dinv not written) on a zero or non-finite pivot.
struct LeafSmem {
  float row[2][BB];
  unsigned cand[2][8];
  int piv[BB], ipiv[BB];
};
__device__ __forceinline__ unsigned pivot_key32(float v, int row) {
  const float a = fabsf(v);
  const unsigned bits = (a == a && a <= 3.4e38f) ? __float_as_uint(a) : 0u;
  return (bits & ~63u) | (unsigned)(BB - 1 - row);  // the low 6 mantissa bits give way to the row
}
__device__ __forceinline__ bool leaf_inverse(const float* Ds, float* Dinv, LeafSmem& L) {
  const int t = threadIdx.x, i = t >> 2, cg = t & 3, lane = t & 31, warp = t >> 5;
  float s[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) s[q] = Ds[i * (BB + 1) + 16 * cg + q];
  bool used = false;
  // pivot of column 0: held by the cg == 0 threads
  {
    const unsigned key = (cg == 0) ? pivot_key32(s[0], i) : 0u;
    const unsigned wk = __reduce_max_sync(0xffffffffu, key);
    if (lane == 0) L.cand[0][warp] = wk;
  }
  __syncthreads();
  unsigned best = 0;
#pragma unroll
  for (int z = 0; z < 8; ++z) best = max(best, L.cand[0][z]);
  bool ok = (best >> 6) != 0;
  int p = BB - 1 - (int)(best & 63u);
  if (t == 0) { L.piv[0] = p; L.ipiv[p] = 0; }
  if (i == p) {
#pragma unroll
    for (int q = 0; q < 16; ++q) L.row[0][16 * cg + q] = s[q];
  }
  __syncthreads();
#pragma unroll 1
  for (int kc = 0; kc < 4 && ok; ++kc) {
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const int k = 16 * kc + kk, buf = k & 1;
      const float ci = __shfl_sync(0xffffffffu, s[kk], (lane & ~3) | kc);
      const float inv = 1.0f / L.row[buf][k];
      const bool prow = (i == p);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = 16 * cg + q;
        const float rj = L.row[buf][j] * inv;
        float v = prow ? rj : fmaf(-ci, rj, s[q]);
        if (j == k) v = prow ? inv : -ci * inv;
        s[q] = v;
      }
      used = used || prow;
      if (k == BB - 1) break;
      // next pivot: column k + 1 is held by the cg == (k + 1) / 16 threads, value s[(k + 1) % 16]
      {
        const int kn = k + 1;
        const float vn = s[(kk + 1) & 15];
        const unsigned key = (cg == (kn >> 4) && !used) ? pivot_key32(vn, i) : 0u;
        const unsigned wk = __reduce_max_sync(0xffffffffu, key);
        if (lane == 0) L.cand[buf ^ 1][warp] = wk;
      }
      __syncthreads();
      best = 0;
#pragma unroll
      for (int z = 0; z < 8; ++z) best = max(best, L.cand[buf ^ 1][z]);
      ok = (best >> 6) != 0;
      p = BB - 1 - (int)(best & 63u);
      if (t == 0) { L.piv[k + 1] = p; L.ipiv[p] = k + 1; }
      if (i == p) {
#pragma unroll
        for (int q = 0; q < 16; ++q) L.row[buf ^ 1][16 * cg + q] = s[q];
      }
      __syncthreads();
      if (!ok) break;
    }
  }
  if (!ok) return false;
  __syncthreads();
  const int ki = L.ipiv[i];
#pragma unroll
  for (int q = 0; q < 16; ++q) Dinv[ki * BB + L.piv[16 * cg + q]] = s[q];
  return true;
}

// The last CTA's look-ahead, during P2 of step k: the next diagonal block
//   D_{k+1} = M[K', K'] - M[K', K] (D_k^{-1} M[K, K'])
// from M as it stands before step k's update (the same values the other CTAs read), in FP32 on the
// CUDA cores, identity beyond its bkn rows; written to Dd[(k + 1) % 2] for the next step's Lhat rows
// and left in shared memory (Ds, row stride 65) for the inverse that follows the barrier.
// sm: shared scratch of >= 4 * 64 * 65 floats (DinvT, M[K][K'] then R_next^T, M[K'][K], Ds).
__device__ __forceinline__ void form_next_block(const BgjArgs& a, int k, int kb, int bk, int kn, int bkn, float* sm) {
  float* DinvT = sm;                   // [s][r] = Dinv[r][s]
  float* Mkn = sm + BB * (BB + 1);     // [s][b] = M[kb + s][kn + b], then R_next^T [b][r]
  float* Lnx = sm + 2 * BB * (BB + 1); // [a][c] = M[kn + a][kb + c]
  float* Ds = sm + 3 * BB * (BB + 1);
  const int t = threadIdx.x;
  {
    constexpr int kV = BB * BB / kThreads;  // elements per thread and array
    float dv[kV], mv[kV], lv[kV];
#pragma unroll
    for (int u = 0; u < kV; ++u) {
      const int e = t + u * kThreads, r = e >> 6, c = e & 63;
      dv[u] = __ldcg(a.Dinv + e);
      mv[u] = (r < bk && c < bkn) ? __ldcg(a.M + (long)(kb + r) * a.ld + kn + c) : 0.0f;
      lv[u] = (r < bkn && c < bk) ? __ldcg(a.M + (long)(kn + r) * a.ld + kb + c) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kV; ++u) {
      const int e = t + u * kThreads, r = e >> 6, c = e & 63;
      DinvT[c * (BB + 1) + r] = dv[u];
      Mkn[r * (BB + 1) + c] = mv[u];
      Lnx[r * (BB + 1) + c] = lv[u];
    }
  }
  __syncthreads();
  const int b = t & 63, g = t >> 6;
  float acc[16];
  // R_next^T[b][r] = sum_s Dinv[r][s] M[kb + s][kn + b], rows r = 16 g .. of thread (b, g)
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
  for (int s_ = 0; s_ < BB; ++s_) {
    const float m = Mkn[s_ * (BB + 1) + b];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = fmaf(DinvT[s_ * (BB + 1) + 16 * g + q], m, acc[q]);
  }
  __syncthreads();  // Mkn is overwritten by R_next^T
#pragma unroll
  for (int q = 0; q < 16; ++q) Mkn[b * (BB + 1) + 16 * g + q] = (16 * g + q < bk) ? acc[q] : 0.0f;
  __syncthreads();
  // D[r][b] = M[kn + r][kn + b] - sum_c Lnx[r][c] R_next^T[b][c]
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
  for (int c = 0; c < BB; ++c) {
    const float rv = Mkn[b * (BB + 1) + c];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = fmaf(Lnx[(16 * g + q) * (BB + 1) + c], rv, acc[q]);
  }
  float* Dd = a.Dd + ((k + 1) & 1) * BB * BB;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int r = 16 * g + q;
    const float v = (r < bkn && b < bkn) ? __ldcg(a.M + (long)(kn + r) * a.ld + kn + b) - acc[q] : (r == b ? 1.0f : 0.0f);
    Ds[r * (BB + 1) + b] = v;
    Dd[r * BB + b] = v;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) k_bgj(BgjArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
  float* sA = reinterpret_cast<float*>(sm);  // Lhat head, then tail, R^T head, tail: 4 x 32 KB
  float* sAt = sA + kOpFloats;
  float* sB = sA + 2 * kOpFloats;
  float* sBt = sA + 3 * kOpFloats;
  float* Ds = sA + 3 * BB * (BB + 1);  // the leader's diagonal block (form_next_block's layout)
  __shared__ LeafSmem L;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = a.n, nb = (n + BB - 1) / BB, nt = (n + BT - 1) / BT;
  const bool leader = blockIdx.x == gridDim.x - 1;
  const int nworkers = gridDim.x - 1;
  unsigned gen = 0;
  if (tid == 0) {
    mbar_init(smem_addr(&mbar), 1);
    failed = 0;
  }
  if (warp == 0) tmem_alloc(&tmem_base, kTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  // Row equilibration: C = R^{-1} (R C) with R = diag(2^-e_i), 2^e_i ~ max_j |C_ij| (exact powers of
  // two, no rounding), so that pivoting inside the diagonal blocks meets rows of one magnitude;
  // C^{-1} = (R C)^{-1} R is recovered by scaling the columns at the end.  One warp per row.
  {
    const int gw = (int)(blockIdx.x * (kThreads / 32)) + warp, nw = (int)gridDim.x * (kThreads / 32);
    for (int i = gw; i < n; i += nw) {
      float* row = a.M + (long)i * a.ld;
      float mx = 0.0f;
      for (int j = lane; j < n; j += 32) mx = fmaxf(mx, fabsf(row[j]));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float sc = (mx > 0.0f && mx <= 3.4e38f) ? exp2f((float)-ilogbf(mx)) : 1.0f;
      for (int j = lane; j < n; j += 32) row[j] *= sc;
      if (lane == 0) a.rscale[i] = sc;
    }
  }
  bool go = grid_barrier(a.sync, gen, a.flags);
  // the first diagonal block: D_0 = M[0:64, 0:64], inverted by the leader
  if (go && leader) {
    const int bk = n < BB ? n : BB;
    for (int e = tid; e < BB * BB; e += kThreads) {
      const int r = e >> 6, c = e & 63;
      const float v = (r < bk && c < bk) ? __ldcg(a.M + (long)r * a.ld + c) : (r == c ? 1.0f : 0.0f);
      Ds[r * (BB + 1) + c] = v;
      a.Dd[e] = v;
    }
    __syncthreads();
    if (!leaf_inverse(Ds, a.Dinv, L) && tid == 0) {
      atomicExch(&a.flags[FLAG_SINGULAR], 1);
      raise_abort(a.sync);
    }
  }
  go = go && grid_barrier(a.sync, gen, a.flags);
  for (int k = 0; k < nb && go; ++k) {
    const int kb = k * BB, bk = (n - kb) < BB ? (n - kb) : BB;
    const int kn = kb + BB, bkn = k + 1 < nb ? ((n - kn) < BB ? (n - kn) : BB) : 0;
    const float* Dcur = a.Dd + (k & 1) * BB * BB;
    // ---- P2: the step's operands (the workers); the leader forms the next diagonal block ----
    if (leader) {
      if (bkn > 0) form_next_block(a, k, kb, bk, kn, bkn, sA);
    } else {
      float* DinvT = sA;         // [s][r] = Dinv[r][s]
      float* Mk = sA + BB * BB;  // [64][16] rows K of a 16-column chunk of M
      {
        float4 d[BB * BB / 4 / kThreads];
#pragma unroll
        for (int u = 0; u < BB * BB / 4 / kThreads; ++u)
          d[u] = __ldcg(reinterpret_cast<const float4*>(a.Dinv) + tid + u * kThreads);
#pragma unroll
        for (int u = 0; u < BB * BB / 4 / kThreads; ++u) {
          const int e = 4 * (tid + u * kThreads), r = e >> 6, c = e & 63;
          DinvT[c * BB + r] = d[u].x;
          DinvT[(c + 1) * BB + r] = d[u].y;
          DinvT[(c + 2) * BB + r] = d[u].z;
          DinvT[(c + 3) * BB + r] = d[u].w;
        }
      }
      // Lhat (rows of every tile, zero beyond n and beyond bk), four elements per thread and round
      const long rows = (long)nt * BT;
      const long gstride = (long)nworkers * kThreads;
      for (long e0 = (long)blockIdx.x * kThreads + tid; e0 < rows * BB; e0 += 4 * gstride) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long e = e0 + u * gstride;
          const int i = (int)(e >> 6), c = (int)(e & 63);
          v[u] = 0.0f;
          if (e < rows * BB && i < n && c < bk) {
            if (i >= kb && i < kb + bk) v[u] = __ldcg(Dcur + (i - kb) * BB + c) - (i - kb == c ? 1.0f : 0.0f);
            else v[u] = __ldcg(a.M + (long)i * a.ld + kb + c);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long e = e0 + u * gstride;
          if (e >= rows * BB) break;
          put_split(a.Lh, a.Lt, op_index((int)(e >> 6), (int)(e & 63)), v[u]);
        }
      }
      __syncthreads();
      // R^T in chunks of 16 columns j: R^T[j][r] = sum_s Dinv[r][s] M[kb + s][j]
      const int nch = (int)(rows / 16);
      const int jj = tid >> 4, r0 = 4 * (tid & 15);
      for (int ch = blockIdx.x; ch < nch; ch += nworkers) {
        const int j0 = 16 * ch;
        {
          float mv[BB * 16 / kThreads];
#pragma unroll
          for (int u = 0; u < BB * 16 / kThreads; ++u) {
            const int e = tid + u * kThreads, s_ = e >> 4, c = e & 15;
            mv[u] = (s_ < bk && j0 + c < n) ? __ldcg(a.M + (long)(kb + s_) * a.ld + j0 + c) : 0.0f;
          }
#pragma unroll
          for (int u = 0; u < BB * 16 / kThreads; ++u) Mk[tid + u * kThreads] = mv[u];
        }
        __syncthreads();
        const int jcol = j0 + jj;
        float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (jcol < n) {
          if (jcol >= kb && jcol < kb + bk) {
#pragma unroll
            for (int u = 0; u < 4; ++u) o[u] = DinvT[(jcol - kb) * BB + r0 + u];
          } else {
            for (int s_ = 0; s_ < BB; ++s_) {
              const float mv = Mk[s_ * 16 + jj];
              const float4 d = *reinterpret_cast<const float4*>(DinvT + s_ * BB + r0);
              o[0] = fmaf(d.x, mv, o[0]);
              o[1] = fmaf(d.y, mv, o[1]);
              o[2] = fmaf(d.z, mv, o[2]);
              o[3] = fmaf(d.w, mv, o[3]);
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (r0 + u >= bk) o[u] = 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) put_split(a.Rh, a.Rt, op_index(jcol, r0 + u), o[u]);
        __syncthreads();
      }
    }
    go = grid_barrier(a.sync, gen, a.flags);
    if (!go) break;
    // ---- P3: tile updates; the leader inverts the next diagonal block meanwhile ----
    if (!leader) {
      for (int tile = blockIdx.x; tile < nt * nt; tile += nworkers) {
        const int TI = tile / nt, TJ = tile - TI * nt;
        {  // the four operand tiles, 16-byte asynchronous copies (L2 only), all in flight at once
          const char* gl = reinterpret_cast<const char*>(a.Lh + (long)TI * kOpFloats);
          const char* gt = reinterpret_cast<const char*>(a.Lt + (long)TI * kOpFloats);
          const char* gr = reinterpret_cast<const char*>(a.Rh + (long)TJ * kOpFloats);
          const char* gs = reinterpret_cast<const char*>(a.Rt + (long)TJ * kOpFloats);
          const uint32_t s0 = smem_addr(sA);
          for (int e = tid; e < kOpBytes / 16; e += kThreads) {
            cp_async16(s0 + 16 * e, gl + 16 * e);
            cp_async16(s0 + kOpBytes + 16 * e, gt + 16 * e);
            cp_async16(s0 + 2 * kOpBytes + 16 * e, gr + 16 * e);
            cp_async16(s0 + 3 * kOpBytes + 16 * e, gs + 16 * e);
          }
          cp_async_wait_all();
        }
        fence_smem_async();
        __syncthreads();
        if (tid == 0) {
          fence_after_sync();
#pragma unroll
          for (int s_ = 0; s_ < BB / 8; ++s_) {
            const uint64_t ah = sdesc(smem_addr(reinterpret_cast<unsigned char*>(sA) + s_ * kSlabBytes));
            const uint64_t at = sdesc(smem_addr(reinterpret_cast<unsigned char*>(sAt) + s_ * kSlabBytes));
            const uint64_t bh = sdesc(smem_addr(reinterpret_cast<unsigned char*>(sB) + s_ * kSlabBytes));
            const uint64_t bt = sdesc(smem_addr(reinterpret_cast<unsigned char*>(sBt) + s_ * kSlabBytes));
            mma_tf32(tmem, ah, bh, kIdesc, s_ > 0 ? 1u : 0u);
            mma_tf32(tmem, ah, bt, kIdesc, 1u);
            mma_tf32(tmem, at, bh, kIdesc, 1u);
          }
          mma_commit(smem_addr(&mbar));
        }
        if (!mbar_wait(smem_addr(&mbar), phase)) failed = 1;
        phase ^= 1u;
        fence_after_sync();
        __syncthreads();
        if (failed) {
          if (tid == 0) {
            atomicExch(&a.flags[FLAG_TIMEOUT], 1);
            mbar_wait(smem_addr(&mbar), phase ^ 1u);  // the MMAs in flight, once more (bounded)
            raise_abort(a.sync);
          }
          break;
        }
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its rows), columns 64 (w / 4) .. + 63 into
        // a shared 128 x 129 tile (the operands are consumed), then every warp updates whole rows of M
        // with coalesced accesses
        {
          float* Ct = sA;
          const int q4 = warp & 3, hh = warp >> 2;
          const int rl = 32 * q4 + lane;
          for (int c8 = 0; c8 < 8; ++c8) {
            const int cl = 64 * hh + 8 * c8;
            uint32_t v[8];
            tmem_ld8(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)cl, v);
#pragma unroll
            for (int u = 0; u < 8; ++u) Ct[rl * (BT + 1) + cl + u] = __uint_as_float(v[u]);
          }
          __syncthreads();
          // warp w updates rows w, w + 8, ..., eight rows per batch: 32 loads in flight per thread
          for (int rb = 0; rb < BT / 8; rb += 8) {
            float cold[8][4];
#pragma unroll
            for (int z = 0; z < 8; ++z) {
              const int i = TI * BT + warp + 8 * (rb + z);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int jcol = TJ * BT + lane + 32 * u;
                const bool in_k = jcol >= kb && jcol < kb + bk;
                cold[z][u] = (i < n && jcol < n && !in_k) ? __ldcg(a.M + (long)i * a.ld + jcol)
                                                          : (i == jcol ? 1.0f : 0.0f);
              }
            }
#pragma unroll
            for (int z = 0; z < 8; ++z) {
              const int rr = warp + 8 * (rb + z), i = TI * BT + rr;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int jl = lane + 32 * u, jcol = TJ * BT + jl;
                if (i < n && jcol < n) a.M[(long)i * a.ld + jcol] = cold[z][u] - Ct[rr * (BT + 1) + jl];
              }
            }
          }
        }
        fence_before_sync();
        __syncthreads();
      }
    } else if (bkn > 0) {
      if (!leaf_inverse(Ds, a.Dinv, L) && tid == 0) {
        atomicExch(&a.flags[FLAG_SINGULAR], 1);
        raise_abort(a.sync);
      }
    }
    go = grid_barrier(a.sync, gen, a.flags);
  }
  if (go)  // C^{-1} = (R C)^{-1} R: column j times the scale of row j
    for (long e = (long)blockIdx.x * kThreads + tid; e < (long)n * n; e += (long)gridDim.x * kThreads) {
      const long i = e / n, j = e - i * n;
      a.M[i * a.ld + j] *= __ldcg(a.rscale + j);
    }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

size_t bgj_smem() { return (size_t)4 * kOpBytes + 1024; }

__global__ void k_bgj_iota(int n, int32_t* p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

}  // namespace

size_t bgj_scratch_bytes(int n) {
  const size_t nt = (size_t)(n + BT - 1) / BT;
  return 4 * nt * kOpBytes + 3 * (size_t)BB * BB * 4 + 4 * (((size_t)n + 63) / 64 * 64) + 256;
}

bool launch_bgj_inverse(int n, float* M, long ld, void* scratch, int32_t* piv, int* flags, int sm_count,
                        cudaStream_t s) {
  if (n <= 0) return true;
  int per_sm = 0;
  const size_t smem = bgj_smem();
  if (cudaFuncSetAttribute(k_bgj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bgj, kThreads, smem) != cudaSuccess || per_sm < 1)
    return false;
  const int nt = (n + BT - 1) / BT;
  int G = sm_count * per_sm;
  if (G > nt * nt + 1) G = nt * nt + 1;
  if (G < 2) return false;
  const size_t ntl = (size_t)nt;
  char* p = static_cast<char*>(scratch);  // 16-byte aligned (operand tiles are copied in 16-byte pieces)
  BgjArgs a;
  a.n = n;
  a.M = M;
  a.ld = ld;
  a.Lh = reinterpret_cast<float*>(p);
  a.Lt = a.Lh + ntl * kOpFloats;
  a.Rh = a.Lt + ntl * kOpFloats;
  a.Rt = a.Rh + ntl * kOpFloats;
  a.Dd = a.Rt + ntl * kOpFloats;
  a.Dinv = a.Dd + 2 * BB * BB;
  a.rscale = a.Dinv + BB * BB;
  a.sync = reinterpret_cast<unsigned*>(a.rscale + ((size_t)n + 63) / 64 * 64);
  a.flags = flags;
  if (cudaMemsetAsync(a.sync, 0, 4 * sizeof(unsigned), s) != cudaSuccess) return false;
  g_launches += 1;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((void*)k_bgj, dim3(G), dim3(kThreads), args, smem, s) != cudaSuccess) return false;
  if (piv) {  // the result is the inverse itself: the identity permutation for the apply
    g_launches += 1;
    k_bgj_iota<<<(n + 255) / 256, 256, 0, s>>>(n, piv);
  }
  return true;
}

}  // namespace ncpadj
