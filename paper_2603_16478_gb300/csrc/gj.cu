// Explicit inverse of a capacitance matrix C = I + h^2 K D (Woodbury, Sec. 4.4) by blocked
// Gauss-Jordan with partial pivoting, organised by column ownership.
//
// Panel p covers columns [p*BP, p*BP + BP).  Block k of the grid owns panels k, k+G, k+2G, ... and
// keeps all n rows of its columns in shared memory for the whole factorisation.  Step p:
//   * the owner of panel p factors it (pivot search among rows not used by earlier panels, one
//     column at a time, the panel in registers), publishes the transformed panel P_p (row-major,
//     BP values per row) and its pivot rows R_p, then raises ready[p];
//   * every block, once ready[p] is set, applies the panel to its other columns j:
//       M'[i][j] = M[i][j] + P_p[i][:] . M[R_p][j]   (i not in R_p),
//       M'[r][j] =           P_p[r][:] . M[R_p][j]   (r in R_p);
//   * the owner of panel p+1 applies step p to that panel first and factors it at once
//     (look-ahead), so the critical path is one panel update + one panel factorisation per step.
// There is no grid-wide barrier: blocks meet only through the ready flags (bounded waits).  After
// the last step the matrix B in A satisfies (C^{-1})[k][piv[k']] = B[piv[k]][k'], the convention of
// the other inverses in this library.  The last block to finish resets the flags to zero.
#include "kernels.cuh"

namespace ncpadj {
namespace {

constexpr int kColsThreads = 512;
constexpr int kColsWarps = kColsThreads / 32;
constexpr long long kColsSpinLimit = 1LL << 21;  // each spin is >= 32 ns of sleep plus two L2 round trips

// sync words: ready[p] per panel, then the abort flag and the count of blocks done
struct ColsSync {
  int* ready;
  int* abort;
  int* done;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Vector accesses to panel rows (BP values, rows BP * sizeof(T) bytes apart): the widest of 16, 8 or
// 4 (8) bytes whose element count W divides BP, so that every access is aligned and inside its row.
template <typename T, int W> struct VecN;
template <> struct VecN<float, 4> { using V = float4; };
template <> struct VecN<float, 2> { using V = float2; };
template <> struct VecN<float, 1> { using V = float; };
template <> struct VecN<double, 2> { using V = double2; };
template <> struct VecN<double, 1> { using V = double; };
template <typename T, int BP> constexpr int vec_width() {
  int w = 16 / (int)sizeof(T);
  while (w > 1 && BP % w != 0) w /= 2;
  return w;
}
template <typename T, int BP> struct RowVec {
  static constexpr int W = vec_width<T, BP>();
  using V = typename VecN<T, W>::V;
};
__device__ __forceinline__ void unpack(const float4& v, float* d) { d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w; }
__device__ __forceinline__ void unpack(const float2& v, float* d) { d[0] = v.x; d[1] = v.y; }
__device__ __forceinline__ void unpack(const float& v, float* d) { d[0] = v; }
__device__ __forceinline__ void unpack(const double2& v, double* d) { d[0] = v.x; d[1] = v.y; }
__device__ __forceinline__ void unpack(const double& v, double* d) { d[0] = v; }
template <typename V, typename T> __device__ __forceinline__ V pack(const T* d);
template <> __device__ __forceinline__ float4 pack<float4, float>(const float* d) { return make_float4(d[0], d[1], d[2], d[3]); }
template <> __device__ __forceinline__ float2 pack<float2, float>(const float* d) { return make_float2(d[0], d[1]); }
template <> __device__ __forceinline__ float pack<float, float>(const float* d) { return d[0]; }
template <> __device__ __forceinline__ double2 pack<double2, double>(const double* d) { return make_double2(d[0], d[1]); }
template <> __device__ __forceinline__ double pack<double, double>(const double* d) { return d[0]; }

template <typename T> __device__ __forceinline__ unsigned abs_key(T v);
template <> __device__ __forceinline__ unsigned abs_key<float>(float v) { return __float_as_uint(fabsf(v)) + 1u; }
template <> __device__ __forceinline__ unsigned abs_key<double>(double v) {
  // order-preserving 32-bit key of |v| (top word of the IEEE bits; ties within the low word are
  // broken by row order, which is deterministic)
  return (unsigned)(__double_as_longlong(fabs(v)) >> 32) + 1u;
}

// SMEM: a block's columns live in shared memory; otherwise in colbuf (global, panel p at p*BP*n)
template <typename T, int BP, int ROWS, bool SMEM>
__global__ void __launch_bounds__(kColsThreads) k_gj_cols(int n, T* __restrict__ A, T* __restrict__ Pbuf,
                                                          T* __restrict__ colbuf, int32_t* __restrict__ piv,
                                                          ColsSync sy, int* flags) {
  const int G = gridDim.x, me = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = (n + BP - 1) / BP;
  const int owned = (np - me + G - 1) / G;  // panels me, me+G, ...
  extern __shared__ __align__(16) unsigned char smraw[];
  T* cols = reinterpret_cast<T*>(smraw);                  // [owned][BP][n], column-major (SMEM)
  T* MR = SMEM ? cols + (size_t)owned * BP * n : cols;    // [BP][owned*BP] old pivot rows
  int* panel_of = reinterpret_cast<int*>(MR + (size_t)BP * owned * BP);  // [n]
  __shared__ unsigned wkey[2][kColsWarps];
  __shared__ int wrowi[2][kColsWarps];
  __shared__ T wval[2][kColsWarps][BP];
  __shared__ int Rcur[BP];
  __shared__ int s_flag;  // 1: stop (abort seen / singular / timeout)
  __shared__ int s_last;
  const int ncol = owned * BP;
  auto pan = [&](int q) -> T* {  // column-major storage of my panel q
    return SMEM ? cols + (size_t)q * BP * n : colbuf + (size_t)(me + q * G) * BP * n;
  };

  // load my columns; rows are spread over threads, BP consecutive columns per row
  for (int q = 0; q < owned; ++q) {
    const int k0 = (me + q * G) * BP;
    for (long e = tid; e < (long)n * BP; e += kColsThreads) {
      const int i = (int)(e / BP), c = (int)(e - (long)i * BP);
      pan(q)[(size_t)c * n + i] = (k0 + c < n) ? A[(size_t)i * n + k0 + c] : T(0);
    }
  }
  for (int i = tid; i < n; i += kColsThreads) panel_of[i] = -1;
  if (tid == 0) s_flag = 0;
  __syncthreads();

  // factor my panel q (global panel p) in registers; false on a zero pivot
  auto factor = [&](int q, int p) -> bool {
    const int k0 = p * BP, bb = min(BP, n - k0);
    T* pc = pan(q);
    T Pr[ROWS][BP];
    bool used[ROWS];
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
      const int i = tid + k * kColsThreads;
      used[k] = i >= n || panel_of[i] >= 0;
#pragma unroll
      for (int c = 0; c < BP; ++c) Pr[k][c] = i < n ? pc[(size_t)c * n + i] : T(0);
    }
    bool ok = true;
#pragma unroll
    for (int jj = 0; jj < BP; ++jj) {
      if (jj < bb && ok) {
        const int buf = jj & 1;
        unsigned key = 0u;
        int bk = -1;
#pragma unroll
        for (int k = 0; k < ROWS; ++k) {
          const unsigned kk = used[k] ? 0u : abs_key<T>(Pr[k][jj]);
          if (kk > key) { key = kk; bk = k; }
        }
        const unsigned mx = __reduce_max_sync(0xffffffffu, key);
        const unsigned bal = __ballot_sync(0xffffffffu, mx != 0u && key == mx);
        if (lane == 0 && mx == 0u) wkey[buf][warp] = 0u;
        if (bal != 0u && lane == __ffs(bal) - 1) {
          wkey[buf][warp] = mx;
          wrowi[buf][warp] = tid + bk * kColsThreads;
#pragma unroll
          for (int k = 0; k < ROWS; ++k)
            if (k == bk)
#pragma unroll
              for (int c = 0; c < BP; ++c) wval[buf][warp][c] = Pr[k][c];
        }
        __syncthreads();
        const unsigned kw = lane < kColsWarps ? wkey[buf][lane] : 0u;
        const unsigned mx2 = __reduce_max_sync(0xffffffffu, kw);
        const unsigned bal2 = __ballot_sync(0xffffffffu, mx2 != 0u && kw == mx2);
        const int w = __ffs(bal2) - 1;
        if (mx2 <= 1u) {  // no unused row, or the largest candidate is zero
          ok = false;
        } else {
          const int r = wrowi[buf][w];
          T prow[BP];
#pragma unroll
          for (int c = 0; c < BP; ++c) prow[c] = wval[buf][w][c];
          const T inv_p = T(1) / prow[jj];
#pragma unroll
          for (int k = 0; k < ROWS; ++k) {
            const int i = tid + k * kColsThreads;
            if (i == r) {
#pragma unroll
              for (int c = 0; c < BP; ++c) Pr[k][c] = (c == jj) ? inv_p : prow[c] * inv_p;
              used[k] = true;
              panel_of[i] = p;
            } else {
              const T m = Pr[k][jj] * inv_p;
#pragma unroll
              for (int c = 0; c < BP; ++c) Pr[k][c] = (c == jj) ? -m : fma(-m, prow[c], Pr[k][c]);
            }
          }
          if (tid == 0) piv[k0 + jj] = r;
        }
      }
    }
    if (!ok) return false;
    // keep the panel (it becomes columns of the inverse) and publish it row-major
    using V = typename RowVec<T, BP>::V;
    constexpr int W = RowVec<T, BP>::W;
#pragma unroll
    for (int k = 0; k < ROWS; ++k) {
      const int i = tid + k * kColsThreads;
      if (i < n) {
#pragma unroll
        for (int c = 0; c < BP; ++c) pc[(size_t)c * n + i] = Pr[k][c];
        V* dst = reinterpret_cast<V*>(Pbuf + ((size_t)p * n + i) * BP);
#pragma unroll
        for (int c = 0; c < BP; c += W) __stcg(dst + c / W, pack<V, T>(&Pr[k][c]));
      }
    }
    return true;
  };

  auto publish = [&](int p, bool ok) {
    __syncthreads();
    if (tid == 0) {
      if (!ok) {
        atomicExch(&flags[FLAG_SINGULAR], 1);
        atomicExch(sy.abort, 1);
        s_flag = 1;
      }
      __threadfence();
      st_release(&sy.ready[p], 1);
    }
    __syncthreads();
  };

  // apply panel p (staged old pivot rows in MR) to my panel q: one row per thread, BP accumulators
  auto update = [&](int q, int p) {
    const int bb = min(BP, n - p * BP);
    using V = typename RowVec<T, BP>::V;
    constexpr int W = RowVec<T, BP>::W;
    T* pc = pan(q);
    const T* mr = MR + q * BP;
    for (int i = tid; i < n; i += kColsThreads) {
      T P[BP];
      const V* src = reinterpret_cast<const V*>(Pbuf + ((size_t)p * n + i) * BP);
#pragma unroll
      for (int c = 0; c < BP; c += W) unpack(__ldcg(src + c / W), &P[c]);
      const bool is_piv = panel_of[i] == p;
      T acc[BP];
#pragma unroll
      for (int c = 0; c < BP; ++c) acc[c] = is_piv ? T(0) : pc[(size_t)c * n + i];
#pragma unroll
      for (int t = 0; t < BP; ++t) {
        if (t < bb) {
          const V* row = reinterpret_cast<const V*>(mr + (size_t)t * ncol);  // broadcast
#pragma unroll
          for (int c = 0; c < BP; c += W) {
            T m[W];
            unpack(row[c / W], m);
#pragma unroll
            for (int u = 0; u < W; ++u) acc[c + u] = fma(P[t], m[u], acc[c + u]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < BP; ++c) pc[(size_t)c * n + i] = acc[c];
    }
  };

  bool stop = false;
  if (me == 0) {  // panel 0 is mine
    const bool ok = factor(0, 0);
    publish(0, ok);
    stop = !ok;
  }
  for (int p = 0; p < np && !stop; ++p) {
    const int k0 = p * BP, bb = min(BP, n - k0);
    const int owner = p % G;
    if (owner != me) {
      if (tid == 0) {
        long long spins = 0;
        int f = 0;
        while ((f = ld_acquire(&sy.ready[p])) == 0 && ld_acquire(sy.abort) == 0) {
          if (++spins > kColsSpinLimit) {
            atomicExch(&flags[FLAG_TIMEOUT], 1);
            atomicExch(sy.abort, 1);
            break;
          }
          __nanosleep(32);
        }
        s_flag = (f == 0 || ld_acquire(sy.abort) != 0) ? 1 : 0;
        __threadfence();
      }
      __syncthreads();
      if (s_flag) break;
    }
    if (tid < bb) {
      const int r = __ldcg(&piv[k0 + tid]);
      Rcur[tid] = r;
      panel_of[r] = p;
    }
    __syncthreads();
    // old pivot rows of my columns (all my panels but p itself)
    for (int e = tid; e < BP * ncol; e += kColsThreads) {
      const int t = e / ncol, jc = e - t * ncol;
      const int q = jc / BP, c = jc - q * BP;
      MR[e] = t < bb ? pan(q)[(size_t)c * n + Rcur[t]] : T(0);
    }
    __syncthreads();
    const int pn = p + 1;
    const int qn = (pn < np && pn % G == me) ? pn / G : -1;
    if (qn >= 0) {  // look-ahead: the next panel first, factor it, publish
      update(qn, p);
      __syncthreads();
      const bool ok = factor(qn, pn);
      publish(pn, ok);
      if (!ok) break;
    }
    for (int q = 0; q < owned; ++q) {
      const int pq = me + q * G;
      if (pq != p && q != qn) update(q, p);
    }
    __syncthreads();
  }
  // write my columns back (row-major) unless the factorisation stopped
  if (tid == 0) s_flag = ld_acquire(sy.abort);
  __syncthreads();
  if (!s_flag) {
    for (int q = 0; q < owned; ++q) {
      const int k0 = (me + q * G) * BP;
      for (long e = tid; e < (long)n * BP; e += kColsThreads) {
        const int i = (int)(e / BP), c = (int)(e - (long)i * BP);
        if (k0 + c < n) A[(size_t)i * n + k0 + c] = pan(q)[(size_t)c * n + i];
      }
    }
  }
  // the last block out clears the flags for the next launch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(sy.done, 1) == G - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int p = tid; p < np; p += kColsThreads) sy.ready[p] = 0;
    __syncthreads();
    if (tid == 0) {
      *sy.abort = 0;
      __threadfence();
      *sy.done = 0;
    }
  }
}

template <typename T, int BP>
size_t cols_smem(int n, int G, bool smem_cols) {
  const int np = (n + BP - 1) / BP;
  const int owned = (np + G - 1) / G;
  return sizeof(T) * ((smem_cols ? (size_t)owned * BP * n : 0) + (size_t)BP * owned * BP) + sizeof(int) * (size_t)n;
}

template <typename T, int BP, int ROWS, bool SMEM>
bool cols_launch(int n, T* A, T* Pbuf, T* colbuf, int32_t* piv, ColsSync sy, int* flags, int G, size_t smem,
                 cudaStream_t s) {
  auto kern = k_gj_cols<T, BP, ROWS, SMEM>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kColsThreads, smem) != cudaSuccess || per_sm < 1)
    return false;
  int nn = n;
  void* args[] = {&nn, &A, &Pbuf, &colbuf, &piv, &sy, &flags};
  // cooperative launch: the blocks wait on one another's flags, so all must be resident
  return cudaLaunchCooperativeKernel((void*)kern, dim3(G), dim3(kColsThreads), args, smem, s) == cudaSuccess;
}

// scratch: kSyncBytes of sync words (ready[np], abort, done) at a fixed place -- every launch
// leaves them zero, whatever its n and type, so one scratch serves inversions of any size --
// then Pbuf [np][n][BP] and colbuf [np][BP][n] (global-column mode)
constexpr int kMaxDim = 32 * kColsThreads;         // n <= 16384
constexpr int kMaxPanels = kMaxDim / 2;            // panels of >= 2 columns
constexpr size_t kSyncBytes = ((sizeof(int) * (kMaxPanels + 4) + 255) / 256) * 256;
template <typename T, int BP>
struct ColsLayout {
  int np;
  size_t pbuf_elems;
  size_t bytes() const { return kSyncBytes + sizeof(T) * 2 * pbuf_elems; }
  explicit ColsLayout(int n) : np((n + BP - 1) / BP), pbuf_elems((size_t)((n + BP - 1) / BP) * BP * n) {}
};

// n in (4096, 16384]: the register panel stays at rows x width <= 64 values with panels of 4 (n <= 8192)
// or 2 columns; columns live in global memory (the matrix exceeds the shared memory of all blocks)
template <typename T, int BPW, int ROWS>
bool cols_invert_wide(int n, T* A, void* scratch, int32_t* piv, int* flags, int sm_count, cudaStream_t s) {
  const ColsLayout<T, BPW> L(n);
  const int G = L.np < sm_count ? L.np : sm_count;
  int* words = static_cast<int*>(scratch);
  T* Pbuf = reinterpret_cast<T*>(static_cast<char*>(scratch) + kSyncBytes);
  ColsSync sy{words, words + kMaxPanels, words + kMaxPanels + 1};
  return cols_launch<T, BPW, ROWS, false>(n, A, Pbuf, Pbuf + L.pbuf_elems, piv, sy, flags, G,
                                            cols_smem<T, BPW>(n, G, false), s);
}

template <typename T, int BP, int BPL>
bool cols_invert(int n, T* A, void* scratch, int32_t* piv, int* flags, int sm_count, cudaStream_t s) {
  constexpr size_t kSmemCap = 200 * 1024;
  const int rows = (n + kColsThreads - 1) / kColsThreads;
  if (rows > 32) return false;
  if constexpr (sizeof(T) == 4) {  // FP64 panels of that height do not fit in registers
    if (rows > 16) return cols_invert_wide<T, 2, 32>(n, A, scratch, piv, flags, sm_count, s);
    if (rows > 8) return cols_invert_wide<T, 4, 16>(n, A, scratch, piv, flags, sm_count, s);
  } else {
    if (rows > 8) return false;
  }
  if (rows > 4) {  // n in (2048, 4096]: narrower panels keep the register panel at 8 x BPL
    const ColsLayout<T, BPL> L(n);
    const int G = L.np < sm_count ? L.np : sm_count;
    int* words = static_cast<int*>(scratch);
    T* Pbuf = reinterpret_cast<T*>(static_cast<char*>(scratch) + kSyncBytes);
    ColsSync sy{words, words + kMaxPanels, words + kMaxPanels + 1};
    const size_t smem = cols_smem<T, BPL>(n, G, false);
    return cols_launch<T, BPL, 8, false>(n, A, Pbuf, Pbuf + L.pbuf_elems, piv, sy, flags, G, smem, s);
  }
  const ColsLayout<T, BP> L(n);
  const int G = L.np < sm_count ? L.np : sm_count;
  int* words = static_cast<int*>(scratch);
  T* Pbuf = reinterpret_cast<T*>(static_cast<char*>(scratch) + kSyncBytes);
  ColsSync sy{words, words + kMaxPanels, words + kMaxPanels + 1};
  T* colbuf = Pbuf + L.pbuf_elems;
  const size_t smem_s = cols_smem<T, BP>(n, G, true);
  if (smem_s <= kSmemCap) {
    if (rows <= 2) return cols_launch<T, BP, 2, true>(n, A, Pbuf, colbuf, piv, sy, flags, G, smem_s, s);
    return cols_launch<T, BP, 4, true>(n, A, Pbuf, colbuf, piv, sy, flags, G, smem_s, s);
  }
  return cols_launch<T, BP, 4, false>(n, A, Pbuf, colbuf, piv, sy, flags, G, cols_smem<T, BP>(n, G, false), s);
}

constexpr int kBP32 = 16, kBP64 = 8;

}  // namespace

namespace {
template <typename T>
__global__ void k_unpermute_inverse(int n, const T* __restrict__ B, const int32_t* __restrict__ piv,
                                    double* __restrict__ out) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)n * n) return;
  const int k = (int)(e / n), kp = (int)(e - (long)k * n);
  out[(size_t)k * n + piv[kp]] = (double)B[(size_t)piv[k] * n + kp];
}
}  // namespace

void launch_unpermute_inverse(int n, const void* B, bool fp32, const int32_t* piv, double* out, cudaStream_t s) {
  g_launches += 1;
  const long ne = (long)n * n;
  const int nb = (int)((ne + 255) / 256);
  if (fp32) k_unpermute_inverse<float><<<nb, 256, 0, s>>>(n, static_cast<const float*>(B), piv, out);
  else k_unpermute_inverse<double><<<nb, 256, 0, s>>>(n, static_cast<const double*>(B), piv, out);
}

size_t gj_cols_scratch_bytes(int n, bool fp32) {
  // the published panels and the column store hold about n^2 values whatever the panel width
  const size_t es = fp32 ? sizeof(float) : sizeof(double);
  return kSyncBytes + 2 * es * (size_t)n * ((size_t)n + 32) + 256;
}
int gj_cols_max_dim() { return kMaxDim; }
int gj_cols_max_dim64() { return 8 * kColsThreads; }
size_t gj_cols_reserved_bytes() { return kSyncBytes; }

// The sync words are cleared before every launch as well: a launch leaves them zero, but a scratch that
// something else wrote (or a fresh allocation) would otherwise let blocks read panels that are not
// published yet, with their stale pivot rows as indices.
bool launch_gj_cols32(int n, float* C, void* scratch, int32_t* piv, int* flags, int sm_count, cudaStream_t s) {
  g_launches += 1;
  if (cudaMemsetAsync(scratch, 0, kSyncBytes, s) != cudaSuccess) return false;
  return cols_invert<float, kBP32, kBP32 / 2>(n, C, scratch, piv, flags, sm_count, s);
}
bool launch_gj_cols64(int n, double* C, void* scratch, int32_t* piv, int* flags, int sm_count, cudaStream_t s) {
  g_launches += 1;
  if (cudaMemsetAsync(scratch, 0, kSyncBytes, s) != cudaSuccess) return false;
  return cols_invert<double, kBP64, kBP64 / 2>(n, C, scratch, piv, flags, sm_count, s);
}

}  // namespace ncpadj
