// Device kernels of the adjoint step and their launch wrappers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ncpadj {

// kernels enqueued by this thread (read and reset by the entry points for their statistics)
extern thread_local long long g_launches;

// status flags written by kernels (int32 slots in Scene::flags)
enum Flag {
  FLAG_INVERTED = 0,   // det F <= 0 in some tet
  FLAG_DOMAIN = 1,     // frictional contact with zero slip and zero tangential force
  FLAG_NONFINITE = 2,  // NaN/Inf seen
  FLAG_SINGULAR = 3,   // zero pivot in the capacitance inversion
  FLAG_TIMEOUT = 4,    // a bounded grid barrier gave up
  FLAG_BARRIER = 5,    // barrier arrival counter
  FLAG_GEN = 6,        // barrier generation
  FLAG_BADINDEX = 7,   // a contact vertex or region id out of range
  FLAG_INFEASIBLE = 8, // forward: a contact outside the local-solve domain (gap <= 0 or zero slip)
  FLAG_TURN = 9,       // forward: a loaded contact's slip turned by more than 60 degrees
  FLAG_COUNT = 12
};

// Scene mask of a batch solve: a kernel given one skips the rows, chunks and contacts of scenes
// whose act[] entry is 0.  sov maps a vertex -- and an elimination position, since every scene's
// positions are its own vertex range -- to its scene.  The default (act = null) masks nothing.
struct Mask {
  const int* act = nullptr;
  const int32_t* sov = nullptr;
#ifdef __CUDACC__
  __device__ __forceinline__ bool on(int v) const { return act == nullptr || act[sov[v]] != 0; }
#endif
};

// ---- element / contact / contraction kernels (elem.cu) ---------------------------------
// constitutive model of a tet (App. B.2); the values are those of NCPADJ_MODEL_*
enum : int8_t { MODEL_NEO_HOOKEAN = 0, MODEL_COROTATIONAL = 1, MODEL_ARAP = 2 };

struct TetArgs {
  int nt;
  const int32_t* tets;
  const double* gvec;  // [nt][12]
  const double* vol;
  const double* mu;
  const double* lam;
  const int32_t* slot;  // [nt][16]
  const double* q;      // [nv][3]
  double h;
  double* bsr;          // [nb][9] (FP64 path) or null
  float* bsr32;         // [nb][9] (mixed path) or null
  double* tetdata;      // [nt][18] contraction tensors
  int* flags;
  const int8_t* model = nullptr;  // [nt] MODEL_* per tet (null: all Neo-Hookean)
};
void launch_tet_assemble64(const TetArgs& a, cudaStream_t s);
void launch_tet_assemble32(const TetArgs& a, cudaStream_t s);

// ---- dense FP32 GEMM on the tensor cores (tc.cu) -------------------------------------------
// C = alpha A B + beta C, row-major with leading dimensions (elements); K >= 1.  split: 3xTF32
// (about FP32 accuracy) instead of plain TF32.  A wait that gives up raises FLAG_TIMEOUT in flags.
struct GemmArgs {
  int M, N, K;
  float alpha, beta;
  const float* A;
  long lda;
  const float* B;
  long ldb;
  float* C;
  long ldc;
  int split;
  int* flags;
};
void launch_tc_gemm(const GemmArgs& g, cudaStream_t s);
size_t tc_gemm_smem(int split);

// M (n x n FP32, row stride ld) <- M^{-1} by blocked Gauss-Jordan elimination in one persistent
// cooperative launch, 64 columns per step, rank-64 updates on the tensor cores (bgj.cu); pivoting
// inside the 64 x 64 diagonal blocks only.  scratch: bgj_scratch_bytes(n) bytes, 16-byte aligned;
// piv (or null) receives the identity permutation, so the Gauss-Jordan apply kernels take the result
// as it is.  A zero pivot raises FLAG_SINGULAR, a wait that gives up FLAG_TIMEOUT.  False if the
// device cannot hold the cooperative grid (nothing launched).
size_t bgj_scratch_bytes(int n);
bool launch_bgj_inverse(int n, float* M, long ld, void* scratch, int32_t* piv, int* flags, int sm_count,
                        cudaStream_t s);
// In-place inverses (FP32 B32 or FP64 B64) of the nsmall blocks ids[] of the capacitance block table
// meta (as launch_cap_apply_all's), one CTA each in one launch, with identity pivots written to piv;
// every listed block must have at most small_inverse_max(fp32) rows and nmax its largest dimension.
int small_inverse_max(bool fp32);
// Delassus blocks D_k (rows [Ds + meta[4 nb + k]], m_k x m_k) and capacitances C_k (FP64 at
// C + meta[k], and FP32 at C32 + meta[k] when C32 is given) of every block in two launches; the
// table has a fifth row, the offsets of the D_k; mmax = the largest m_k
void launch_cap_form_all(int nb, int mmax, const int64_t* meta, const int32_t* cvertex, const int32_t* iperm,
                         const int64_t* St_ptr, const int32_t* St_col, const double* St_val, double* Ds,
                         const double* frame, const double* cdata, double h, int transpose, double* C, float* C32,
                         cudaStream_t s);
void launch_small_inverse(int nsmall, const int32_t* ids, int nb, const int64_t* meta, int nmax, float* B32,
                          double* B64, int32_t* piv, int* flags, cudaStream_t s);
// x_k = B_k y_k (both pivot permutations, as launch_gj_apply*) for all nb capacitance blocks in one
// launch; meta: int64 [4][nb] = element offset of B_k, offset 3 c0_k of its rows in y/x (and piv),
// dimension n_k <= nmax, scene; B32 (FP32 inverses) or B64; act (nullable): skip blocks of idle scenes;
// accumulate: x_k += B_k y_k
void launch_cap_apply_all(int nb, int nmax, const int64_t* meta, const float* B32, const double* B64,
                          const int32_t* piv, const double* y, double* x, const int* act, cudaStream_t s,
                          bool accumulate = false);
// r_k = y_k - C_k x_k in FP64 for every block of the same table, C_k the capacitance itself (unpermuted,
// at C + meta[k]), x_k in natural order: the residual of a refinement step of the capacitance solve
void launch_cap_resid_all(int nb, int nmax, const int64_t* meta, const double* C, const double* y, const double* x,
                          double* r, const int* act, cudaStream_t s);
// x[0..n) = v
void launch_fill(long n, double v, double* x, cudaStream_t s);

// ---- triangle (shell) elements and isometric bending (shell.cu) ---------------------------
// TetArgs with the triangle layout: tets [nt][3], gvec [nt][6] (2-vectors g_0..g_2), slot [nt][9],
// tetdata [nt][12] (P_mu, P_lam as 3 x 2 row-major), vol = area * thickness
void launch_tri_assemble64(const TetArgs& a, cudaStream_t s);
void launch_tri_assemble32(const TetArgs& a, cudaStream_t s);
void launch_tri_force(int nt, const int32_t* tris, const double* gvec, const double* vol, const double* mu,
                      const double* lam, const int8_t* model, const double* q, double h, double* R, int* flags,
                      cudaStream_t s);
// hinges: idx [ne][4] vertices, coef [ne][5] = (K_0..K_3, 3/(A_1+A_2)), kb [ne] stiffness of the
// hinge's mesh, slot [ne][16] block slots of the vertex pairs
void launch_bend_blocks(int ne, const int32_t* idx, const double* coef, const double* kb, const int32_t* slot,
                        double h, double* bsr, float* bsr32, cudaStream_t s);
void launch_bend_force(int ne, const int32_t* idx, const double* coef, const double* kb, const double* q, double h,
                       double* R, cudaStream_t s);
// out[s] = dL/dk_b of mesh s = -h^2 z^T Q_s q over its hinges [eoff[s], eoff[s+1])
void launch_bend_grad(int n_scenes, const int32_t* eoff, const int32_t* idx, const double* coef, const double* q,
                      const double* z, double h, double* out, cudaStream_t s);

struct ContactArgs {
  int nc;
  const int32_t* vertex;
  const double* frame;   // [nc][9]
  const double* d_n;
  const double* d_f;     // [nc][2] or null
  const double* mu;
  const double* lambda;  // [nc][3]
  const double* q;
  const double* q_prev;
  const int32_t* diag_slot;
  double eps, h;
  int transpose;         // 1: add K^T (adjoint matrix script_A^T), 0: add K (Newton matrix script_A)
  double* bsr;           // add h^2 F^T K^T F into diagonal blocks (FP64) or null
  float* bsr32;          // or FP32
  double* cdata;         // [nc][12] K (frame coords, row-major), k_mu
  int* flags;
};
void launch_contact_blocks(const ContactArgs& a, cudaStream_t s);
// flags FLAG_BADINDEX if any contact vertex is outside [0, nv) or region outside [0, nreg)
void launch_check_contacts(int nc, const int32_t* vertex, const int32_t* region, int nv, int nreg, int* flags,
                           cudaStream_t s);

void launch_bsr_init(int nv, int nb, const int32_t* diag_slot, const double* mass, double* bsr,
                     float* bsr32, cudaStream_t s);

struct ContractArgs {
  int nv, nt, nc;
  double h;
  const double* z;
  const double* mass;
  const double* dL_dv;   // may be null
  const int32_t* tets;
  const double* gvec;
  const double* tetdata;
  const double* lame_d;  // [nt][4]
  const int32_t* cvertex;
  const double* frame;
  const double* cdata;
  const int32_t* region;  // may be null
  double* dL_dq_prev;
  double* dL_dv_prev;
  double* dL_dfext;
  double* dL_dE;
  double* dL_dnu;
  double* dL_dmu;         // [n_regions] (zeroed by the caller)
  double* dL_dmu_contact; // [nc]
};
void launch_contractions(const ContractArgs& a, cudaStream_t s);  // the tet part runs when nt > 0
void launch_contract_tri(const ContractArgs& a, cudaStream_t s);  // dL/dE, dL/dnu of triangles
// batch scenes: scene id of every contact; per-scene sums of squares of a DOF vector (sq zeroed by
// the caller); x[i] *= scale[scene_of_vertex[i / 3]]
void launch_contact_scene(int nc, const int32_t* cvertex, const int32_t* scene_of_vertex, int32_t* out, cudaStream_t s);
void launch_scene_sq(int nv, const double* x, const int32_t* scene_of_vertex, double* sq, cudaStream_t s);
void launch_scale_by_scene(int nv, double* x, const int32_t* scene_of_vertex, const double* scale, cudaStream_t s);

// ---- forward step (elem.cu) ----------------------------------------------------------------
// qt = q_prev + h v_prev + h^2 (g + f_ext / m)
// f += -sum_i V_i G_i^T vec(a_i d_i d_i^T) (actuation force; f holds f_ext on entry)
void launch_act_force(int nt, const int32_t* tets, const double* gvec, const double* vol, const float* act,
                      const double* fibre, double* f, cudaStream_t s);
// out[i] = -h^2 V_i d_i^T Z_i d_i with Z_i = unvec(G_i z) (FP32 output)
void launch_act_grad(int nt, const int32_t* tets, const double* gvec, const double* vol, const double* fibre,
                     const double* z, double h, float* out, cudaStream_t s);
void launch_predict(int nv, const double* q_prev, const double* v_prev, const double* f_ext, const double* mass,
                    double g0, double g1, double g2, double h, double* qt, cudaStream_t s);
// q[v_c] += max(0, gap0 - delta_n) n_c  (start point inside the local-solve domain)
void launch_lift(int nc, const int32_t* vertex, const double* frame, const double* d_n, double gap0, double* q,
                 const double* q_prev, const double* d_f, cudaStream_t s);
// R = M (q - qt)
void launch_inertia(int nv, const double* mass, const double* q, const double* qt, double* R, cudaStream_t s);
// R[v_a] += h^2 w_i (F - p(F)) g_a  (elastic force of Eq. internal)
// bilateral bindings on single vertices (Eq. binding): index / compliance check (FLAG_BADINDEX),
// h^2 / E_b I_3 into the diagonal blocks, the residual's binding force, and dL/dd_b, dL/dE_b
void launch_check_bindings(int nb, const int32_t* vertex, const double* compliance, int nv, int* flags,
                           cudaStream_t s);
void launch_binding_blocks(int nb, const int32_t* vertex, const double* compliance, const int32_t* diag_slot,
                           double h, double* bsr, float* bsr32, cudaStream_t s);
void launch_binding_force(int nb, const int32_t* vertex, const double* target, const double* compliance,
                          const double* q, double h, double* R, cudaStream_t s);
void launch_binding_grad(int nb, const int32_t* vertex, const double* target, const double* compliance,
                         const double* q, const double* z, double h, double* d_target, double* d_compliance,
                         cudaStream_t s);
// the same for points inside tets (tet [nb], bary [nb][4]; blocks through the element->slot map)
void launch_check_bindings_bary(int nb, const int32_t* tet, const double* bary, const double* compliance, int nt,
                                int* flags, cudaStream_t s);
void launch_binding_blocks_bary(int nb, const int32_t* tet, const double* bary, const double* compliance,
                                const int32_t* slot, double h, double* bsr, float* bsr32, cudaStream_t s);
void launch_binding_force_bary(int nb, const int32_t* tet, const int32_t* tets, const double* bary,
                               const double* target, const double* compliance, const double* q, double h, double* R,
                               cudaStream_t s);
void launch_binding_grad_bary(int nb, const int32_t* tet, const int32_t* tets, const double* bary,
                              const double* target, const double* compliance, const double* q, const double* z,
                              double h, double* d_target, double* d_compliance, cudaStream_t s);
void launch_tet_force(int nt, const int32_t* tets, const double* gvec, const double* vol, const double* mu,
                      const double* lam, const int8_t* model, const double* q, double h, double* R, int* flags,
                      cudaStream_t s);
// exact local solution of the contact equations at q: lambda_n = eps^2/delta_n,
// gamma = mu lambda_n - eps^2/||delta_f||; writes lambda (frame coords), slips, loaded mask, and
// R[v] -= h^2 F^T lambda
void launch_local_contact(const ContactArgs& a, double* lambda, double* slip, int* loaded, double* R,
                          cudaStream_t s);
// FLAG_TURN if a loaded contact's slip turned by more than 60 degrees from slip_old
void launch_turn_check(int nc, const double* slip_old, const double* slip_new, const int* loaded, int* flags,
                       const int32_t* cvertex, double* R, cudaStream_t s);
// q_out = q + t[scene(v)] dx per vertex (per-scene step lengths of a batch)
void launch_step_by_scene(int nv, const double* q, const double* dx, const int32_t* sov, const double* t,
                          double* q_out, cudaStream_t s);

// ---- linear algebra (linalg.cu) ---------------------------------------------------------
// y = B x for the 3x3-block matrix (FP64)
void launch_bsr_spmv(int nv, const int32_t* row_ptr, const int32_t* col, const double* val,
                     const double* x, double* y, cudaStream_t s, const Mask& mk = Mask{});
void launch_bsr_spmv32(int nv, const int32_t* row_ptr, const int32_t* col, const float* val,
                       const double* x, double* y, cudaStream_t s, const Mask& mk = Mask{});
// y = B x for FP32 block values with x as double-float pairs (hi, lo) [3 nv], double-float
// arithmetic (FP64-class accuracy) on the FP32 pipes; with jp, y is V_{j+1} = ybase + (*jp + 1) yld
void launch_bsr_spmv_ff(int nv, const int32_t* rp, const int32_t* col, const float* val, const float2* x2,
                        double* ybase, long yld, const int* jp, cudaStream_t s, const Mask& mk = Mask{});
// x2 = double-float pairs of x (n values)
void launch_split(int n, const double* x, float2* x2, cudaStream_t s);
// inverse of the scalar diagonal of the block matrix
void launch_diag_inv(int nv, const int32_t* diag_slot, const double* val, const float* val32, double* dinv,
                     cudaStream_t s);

// A^{-1} x = P^T S^T S P x for 3 right-hand sides ([nv][3]); w is [nv][3] scratch
struct SinvArgs {
  int nv;
  const int64_t* S_ptr;
  const int32_t* S_c0;    // [nS] first column (position) of each chunk of S: rows of S are
                          // contiguous column ranges, so no per-entry index is kept
  const double* S_val;
  const int64_t* St_ptr;
  const int32_t* St_col;  // positions
  const double* St_val;
  const int32_t* perm;
  // chunks of at most `chunk` entries (128, 256 or 512) of the rows of S and S^T
  int nS, nSt;
  const int32_t *S_crow, *St_crow;
  const int64_t *S_cbeg, *S_cend, *St_cbeg, *St_cend;
  const float *S_val32 = nullptr, *St_val32 = nullptr;  // FP32 copies (mixed precision)
  // scratch [nv][3]: x permuted to elimination (position) order before the product with S, whose
  // columns are positions -- row p of S covers the descendants of p, a contiguous position range,
  // so the product gathers x contiguously
  double* xpos = nullptr;
  float* xpos32 = nullptr;
  int chunk = 256;
};
void launch_ainv(const SinvArgs& a, const double* x, double* w, double* y, cudaStream_t s);
// Step-indexed forms for a captured GMRES step (j = *jp on the device; V_{j+1} = V + (j + 1) ld):
//   w = S P V_j (zeroed first; FP32 values into w32 when given)
void launch_sinv_half1_idx(const SinvArgs& a, const double* xbase, long xld, const int* jp, double* w, float* w32,
                           cudaStream_t s, const Mask& mk = Mask{});
//   V_{j+1} = A x (block matrix, FP64 or FP32 values)
void launch_bsr_spmv_idx(int nv, const int32_t* rp, const int32_t* col, const double* val, const float* val32,
                         const double* x, double* ybase, long yld, const int* jp, cudaStream_t s,
                         const Mask& mk = Mask{});
//   out[k] = V_k . V_{j+1}, k <= j (or, with self, out[0] = |V_{j+1}|^2); mmax = largest j + 1
void launch_multi_dot_idx(int n, int mmax, const double* V, long ld, const int* jp, bool self, double* partial,
                          double* out, cudaStream_t s);
//   V_{j+1} -= sum_k coef[k] V_k ;  V_{j+1} /= sqrt(*nrm2) (norm to *h_slot)
void launch_multi_axpy_idx(int n, const double* V, long ld, const int* jp, const double* coef, double* Vw,
                           cudaStream_t s);
void launch_normalize_idx(int n, double* V, long ld, const int* jp, const double* nrm2, double* h_slot, cudaStream_t s);
//   gs[0..len) to host-mapped slot j % 2, then *jp = j + 1
// Y + (*jp) * ld <- x (n values; *jp read on the device)
void launch_copy_idx(int n, const double* x, double* Y, long ld, const int* jp, cudaStream_t s);
void launch_export_step(const double* gs, int len, double* host_slots, int* jp, cudaStream_t s);
// the two halves of A^{-1} = P^T S^T S P: w = S P x (position space, zeroed first), y = P^T S^T w
void launch_sinv_half1(const SinvArgs& a, const double* x, double* w, cudaStream_t s, const Mask& mk = Mask{});
void launch_sinv_half2(const SinvArgs& a, const double* w, double* y, cudaStream_t s, const Mask& mk = Mask{});
void launch_sinv_half1_32(const SinvArgs& a, const double* x, float* w32, cudaStream_t s, const Mask& mk = Mask{});
void launch_sinv_half2_32(const SinvArgs& a, const float* w32, double* y, cudaStream_t s, const Mask& mk = Mask{});
// s_c = K'_c F_c (A^{-1} x)_{v_c} from w = S P x, along the elimination-tree paths of the contact
// vertices (w: double, or w32 float with the FP32 values when w32 is not null)
void launch_path_gather(int nc, const int32_t* cvertex, const int32_t* iperm, const SinvArgs& a, const double* w,
                        const float* w32, const double* frame, const double* cdata, int transpose, double* sc,
                        cudaStream_t s, const Mask& mk = Mask{});
// w += coef S P J^T t (contact forces t in frame coordinates), along the same paths
void launch_path_scatter(int nc, const int32_t* cvertex, const int32_t* iperm, const SinvArgs& a, const double* frame,
                         const double* t, double coef, double* w, float* w32, cudaStream_t s,
                         const Mask& mk = Mask{});
// the same with FP32 values and intermediate (x32, w32 [nv][3] float scratch); y accumulated in FP64
void launch_ainv32(const SinvArgs& a, const double* x, float* x32, float* w32, double* y, cudaStream_t s);

// score[c] = h^2 |K_c|_F (A_s^{-1})_{v_c v_c}: the distance of contact c's capacitance rows from the
// identity (contacts far below 1 are left out of the capacitance set)
void launch_contact_score(int nc, const int32_t* cvertex, const int32_t* iperm, const int64_t* St_ptr,
                          const double* St_val, const double* cdata, double h, double* score, cudaStream_t s);
// vertex, frame and K / k_mu of the contacts idx[0..nk) into compact arrays
void launch_gather_contacts(int nk, const int32_t* idx, const int32_t* vertex, const double* frame,
                            const double* cdata, int32_t* ov, double* of, double* oc, cudaStream_t s);
// single-vertex bindings as capacitance members after the first `off`: vertex, identity frame,
// K = I / E_b
void launch_binding_capdata(int nb, const int32_t* vertex, const double* compliance, int off, int32_t* ov,
                            double* of, double* oc, cudaStream_t s);
// Delassus of the contact vertices: Ds[a][b] = (A_s^{-1})_{v_a v_b}
void launch_delassus(int nc, const int32_t* cvertex, const int32_t* iperm, const int64_t* St_ptr,
                     const int32_t* St_col, const double* St_val, double* Ds, cudaStream_t s);
// capacitance C = I + h^2 K^T D (3nc x 3nc, row-major)
void launch_cap_form(int nc, const double* Ds, const double* frame, const double* cdata, double h, int transpose,
                     double* C, cudaStream_t s);
// Column-owned blocked Gauss-Jordan with partial pivoting (gj.cu): C is swept in place into B, the
// pivot rows go to piv (apply with launch_gj_apply*).  scratch
// holds gj_cols_scratch_bytes(n) bytes and must be zero before its first use (the kernel leaves its
// flags zero).  Returns false without launching when n > gj_cols_max_dim() or the launch is refused.
size_t gj_cols_scratch_bytes(int n, bool fp32);
int gj_cols_max_dim();    // FP32
int gj_cols_max_dim64();  // FP64
// the first gj_cols_reserved_bytes() of that scratch hold its flags: other users of the same
// buffer must start after them
size_t gj_cols_reserved_bytes();
bool launch_gj_cols32(int n, float* C, void* scratch, int32_t* piv, int* flags, int sm_count, cudaStream_t s);
bool launch_gj_cols64(int n, double* C, void* scratch, int32_t* piv, int* flags, int sm_count, cudaStream_t s);
// out[k][piv[k']] = B[piv[k]][k']: the plain inverse from the Gauss-Jordan result B (float or double)
void launch_unpermute_inverse(int n, const void* B, bool fp32, const int32_t* piv, double* out, cudaStream_t s);
// (act, scene): the launch does nothing while act[scene] is 0 (batch solves)
void launch_gj_apply32(int n, const float* B, const int32_t* piv, const double* y, double* ytmp, double* x,
                       cudaStream_t s, const int* act = nullptr, int scene = 0);
void launch_convert_f32(long n, const double* x, float* y, cudaStream_t s);
// x = C^{-1} y with the swept matrix B and pivot rows: x_k = B[piv_k] . y[piv]
void launch_gj_apply(int n, const double* B, const int32_t* piv, const double* y, double* ytmp, double* x,
                     cudaStream_t s, const int* act = nullptr, int scene = 0);

// vector kernels
void launch_axpby(int n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s);
void launch_rhs(int n, const double* dL_dq, const double* dL_dv, double inv_h, double* b, cudaStream_t s);
void launch_mul(int n, const double* a, const double* b, double* y, cudaStream_t s);
// out[k] = sum_i V_k[i] w[i], k < nvec <= kMaxDotVectors (vectors of length n, stride ld); partial is a
// scratch of dot_scratch_bytes() whose trailing counters must be zero before the first use (the
// kernel leaves them zero)
constexpr int kMaxDotVectors = 520;
inline size_t dot_scratch_bytes() { return sizeof(double) * 64 * kMaxDotVectors + sizeof(unsigned) * kMaxDotVectors; }
void launch_multi_dot(int n, int nvec, const double* V, long ld, const double* w, double* partial, double* out,
                      cudaStream_t s);
// w -= sum_k coef[k] V_k (coef on device); if add_to != null also add_to[k] += coef[k]
void launch_multi_axpy(int n, int nvec, const double* V, long ld, const double* coef, double* w,
                       cudaStream_t s);
// y = sum_k coef[k] V_k
void launch_combine(int n, int nvec, const double* V, long ld, const double* coef, double* y, cudaStream_t s);
// v_out = w / nrm (nrm on device); writes nrm into H slot too
void launch_normalize(int n, const double* w, const double* nrm2, double* v_out, double* h_slot, cudaStream_t s);
// CG scalar updates
void launch_cg_alpha(const double* rz, const double* pAp, double* alpha, cudaStream_t s);
void launch_cg_update_xr(int n, const double* alpha, const double* p, const double* Ap, double* x, double* r,
                         cudaStream_t s);
void launch_cg_update_p(int n, const double* rz_new, const double* rz_old, const double* z, double* p,
                        cudaStream_t s);
void launch_copy_scalar(const double* src, double* dst, cudaStream_t s);
void launch_nonfinite_check(int n, const double* x, int* flags, cudaStream_t s);


// ---- batched per-scene GMRES (batch.cu) ------------------------------------------------------
constexpr int kMaxRestart = 512;  // largest GMRES restart length (ncpadj_options.gmres_restart)
// Tiles of a batch scene's DOF range [0, 3 nv): tile t covers [beg[t], end[t]) of scene scene[t]
// (never two scenes); the tiles of scene s are t0[s] .. t0[s+1]-1.
struct SegTiles {
  int n = 0;
  const int32_t* scene = nullptr;
  const int32_t* beg = nullptr;
  const int32_t* end = nullptr;
  const int32_t* t0 = nullptr;
};
constexpr int kSegTile = 2048;
// Step j = *jp of every active scene's Arnoldi process (V_{j+1} = V + (j + 1) ld):
//   gsb[s][goff + k] = V_k . V_{j+1} (k <= j), or with self gsb[s][goff] = |V_{j+1}|^2.
//   partial: m x T.n doubles; cnt: K zero counters per scene (K >= m + 3; slots m + 1, m + 2 are the
//   self dot and launch_seg_sq's), left zero.
void launch_seg_dot_step(const SegTiles& T, const double* V, long ld, const int* jp, int m, bool self, const int* act,
                         double* partial, unsigned* cnt, int K, double* gsb, int gstride, int goff, cudaStream_t s);
//   out[s] = |x_s|^2 for the scenes with mask[s]
void launch_seg_sq(const SegTiles& T, const double* x, const int* mask, double* partial, unsigned* cnt, int K, int slot,
                   double* out, cudaStream_t s);
//   V_{j+1} -= sum_{k <= j} gsb[s][goff + k] V_k ;  V_{j+1} /= sqrt(gsb[s][noff])
void launch_seg_axpy_step(const SegTiles& T, double* V, long ld, const int* jp, int m, const int* act,
                          const double* gsb, int gstride, int goff, cudaStream_t s);
void launch_seg_normalize_step(const SegTiles& T, double* V, long ld, const int* jp, int m, const int* act,
                               const double* gsb, int gstride, int noff, cudaStream_t s);
//   dst = src or d .* src (d not null), src / dst offset by j ld when *_idx; with split (not null)
//   also split[i] = the double-float pair of dst[i]
void launch_seg_copy_step(const SegTiles& T, const double* src, bool src_idx, double* dst, bool dst_idx, long ld,
                          const int* jp, int m, const int* act, const double* d, cudaStream_t s,
                          float2* split = nullptr);
//   Hessenberg column j, Givens rotations and stopping test of every active scene; nact[j] (host
//   mapped) = scenes still active; *jp = j + 1
void launch_seg_givens(int ns, int* jp, int m, int* act, const double* gsb, int gstride, double* H, double* cs,
                       double* sn, double* g, int* kk, int* iters, const double* tol, int maxit, int* nact,
                       cudaStream_t s);
// end of a cycle: y_s = H_s^{-1} g_s, x += Z y_s, r = b - w, restart (see batch.cu)
void launch_seg_backsolve(int ns, int m, const int* cyc, const int* kk, const double* H, const double* g, double* y,
                          cudaStream_t s);
void launch_seg_combine(const SegTiles& T, const double* Z, long ld, int m, const int* cyc, const int* kk,
                        const double* y, double* x, cudaStream_t s);
void launch_seg_resid(const SegTiles& T, const double* b, const double* w, const int* mask, double* r, cudaStream_t s);
void launch_seg_restart(int ns, int m, bool first, int* cyc, int* act, int* done, int* kk, const int* iters,
                        int maxit, const double* rr, double* bnorm, double* tol, double rtol, double* relres,
                        double* g, int* jp, int* flags, int* notdone, cudaStream_t s);
void launch_seg_start(const SegTiles& T, const double* r, const int* act, const double* g, int m, double* V,
                      cudaStream_t s);
void launch_seg_init(int ns, int* cyc, int* done, int* iters, cudaStream_t s);
// table-driven copies (one block per entry): FP64 arrays, int32 ids plus an offset (a null source
// gives the offset alone), FP32 arrays
void launch_gather_f64(int nent, const double* const* src, double* const* dst, const int64_t* cnt, cudaStream_t s);
void launch_gather_ids(int nent, const int32_t* const* src, int32_t* const* dst, const int64_t* cnt,
                       const int32_t* add, cudaStream_t s);
void launch_gather_f32(int nent, const float* const* src, float* const* dst, const int64_t* cnt, cudaStream_t s);
// FLAG_BADINDEX unless contact c's vertex and region (already offset) lie in its own scene's ranges
// (c in [coff[s], coff[s+1]) belongs to scene s; voff, roff: [ns + 1] vertex and region offsets)
void launch_check_batch_ids(int nc, const int32_t* vertex, const int32_t* region, int ns, const int32_t* coff,
                            const int32_t* voff, const int32_t* roff, int* flags, cudaStream_t s);

}  // namespace ncpadj
