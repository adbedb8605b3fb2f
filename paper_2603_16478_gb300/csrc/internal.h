// Internal declarations of the ncpadj library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ncpadj.h"

namespace ncpadj {

// ------------------------------------------------------------------------------------------
// error plumbing
// ------------------------------------------------------------------------------------------
void set_error(const std::string& msg);
struct Error {
  ncpadj_status status;
  std::string msg;
};
#define NCPADJ_CUDA_TRY(expr)                                                              \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::ncpadj::Error{NCPADJ_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define NCPADJ_REQUIRE(cond, msg) \
  do {                            \
    if (!(cond)) throw ::ncpadj::Error{NCPADJ_ERR_INVALID_ARG, msg}; \
  } while (0)

// device buffer (grow-only)
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void ensure(size_t n);
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
  ~DevBuf() { release(); }
};

// ------------------------------------------------------------------------------------------
// host-side factorisation of the scalar elastic matrix (factor.cpp)
// ------------------------------------------------------------------------------------------
struct CsrD {
  int n = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

struct ElasticFactor {
  int n = 0;
  std::vector<int32_t> perm;   // perm[i] = original vertex at elimination position i
  std::vector<int32_t> iperm;  // iperm[v] = elimination position of vertex v
  std::vector<int32_t> parent; // elimination tree (position space), -1 at roots
  int64_t nnz_L = 0;
  CsrD S;   // S = L^{-1} by rows, position space (row i: columns j <= i, descendants of i)
  CsrD St;  // S^T by rows = columns of S (row j: entries i >= j on the etree path from j)
};

// A_s given as a symmetric CSR (both triangles) in original vertex numbering.
// xyz [n][3] vertex coordinates drive the nested-dissection ordering.
void factor_elastic(const CsrD& As, const double* xyz, ElasticFactor& out);

// ------------------------------------------------------------------------------------------
// device data of a scene
// ------------------------------------------------------------------------------------------
struct Scene {
  int nv = 0, nt = 0, nb = 0;
  int n_scenes = 1;                 // meshes in the (batch) scene
  std::vector<int> voff, toff;      // vertex / tet offsets of each mesh [n_scenes + 1]
  DevBuf scene_of_vertex;           // int32 [nv]
  DevBuf sceneval;                  // per-scene scale factors (batch adjoints)
  DevBuf cscene;                    // int32 [nc]: mesh of each contact (batch scenes)
  double h = 0, density = 0;
  // host copies
  std::vector<double> mass;  // [nv]
  // device
  DevBuf tets;      // int32 [nt][4]
  DevBuf gvec;      // double [nt][12]  g_0..g_3 (rows of the 4x3 gradient operator)
  DevBuf vol;       // double [nt]
  DevBuf mu, lam;   // double [nt]  Lame parameters
  DevBuf lame_d;    // double [nt][4] dmu/dE, dlam/dE, dmu/dnu, dlam/dnu
  DevBuf massd;     // double [nv]
  DevBuf row_ptr;   // int32 [nv+1]  block pattern of script_A
  DevBuf col;       // int32 [nb]
  DevBuf slot;      // int32 [nt][16] block slot of (a, b)
  DevBuf diag_slot; // int32 [nv]
  // elastic factor (position space), device copies
  DevBuf perm, iperm;          // int32 [nv]
  DevBuf S_ptr, S_c0, S_val;   // rows of S (position space; each a contiguous column range),
                               // S_c0: the first column of each chunk
  DevBuf St_ptr, St_col, St_val;  // rows of S^T; St_col in position space
  DevBuf S_val32, St_val32;       // FP32 copies of the values (mixed precision)
  DevBuf S_crow, S_cbeg, S_cend, St_crow, St_cbeg, St_cend;  // row chunks (<= 256 entries)
  int nS_chunks = 0, nSt_chunks = 0;
  int chunk = 256;  // entries per chunk of the A^{-1} product (128, 256 or 512; ncpadj_scene_set_chunk)
  int64_t nnz_S = 0;
  int64_t nnz_L = 0;
  double ms_factor = 0;
  // shells (nvpe = 3): the triangles take the tet arrays above with their own layout (tets [nt][3],
  // gvec [nt][6], slot [nt][9], tetdata [nt][12], vol = area * thickness); bending hinges:
  int nvpe = 4;                     // vertices per element
  int n_bend = 0;                   // hinges (interior edges) over the whole scene
  DevBuf bend_idx;                  // int32 [n_bend][4] vertices (edge, then the two opposite)
  DevBuf bend_coef;                 // double [n_bend][5] cotangent stencil K_0..K_3, 3/(A_1+A_2)
  DevBuf bend_kb;                   // double [n_bend] bending stiffness of the hinge's mesh
  DevBuf bend_slot;                 // int32 [n_bend][16] block slots of the vertex pairs
  DevBuf bend_eoff;                 // int32 [n_scenes + 1] hinge offsets of each mesh
  // host copies of the meshes (for a refactor with new materials) and the current material
  std::vector<std::vector<double>> geo_pos;
  std::vector<std::vector<int32_t>> geo_tets;
  std::vector<double> geo_density, geo_thickness;
  std::vector<double> mat_E, mat_nu;  // [nt]
  std::vector<double> mat_bend;       // [n_scenes] (shells)
  std::vector<int64_t> St_ptr_h;  // host copy (Delassus pair scheduling)
  std::vector<int64_t> S_ptr_h;   // host copies of S's row pointers and each row's first column (chunking)
  std::vector<int32_t> S_first_h;

  // per-call workspace
  DevBuf bsr64, bsr32;            // block values
  DevBuf tetdata;                 // double [nt][18]  P_mu, P_lam contraction tensors
  DevBuf cdata;                   // double [nc][16]  per-contact K (9), kmu (3), M_a pieces
  DevBuf c_in;                    // staging of contact inputs for host-memory calls
  DevBuf vecs;                    // Krylov vectors
  DevBuf cap, capw;               // capacitance matrix / inverse and the Gauss-Jordan scratch (sync words zero)
  DevBuf recw;                    // scratch of the tensor-core capacitance inverse (separate from capw)
  DevBuf capmeta;                 // int64 [4][blocks]: the capacitance block table of the one-launch apply
  DevBuf capres;                  // residual of the refined capacitance solve (NCPADJ_REFINED) [3 contacts]
  DevBuf capchk;                  // probe, product and residual of the tensor-core inverse check [3][3 contacts]
  DevBuf capids;                  // int32: the blocks small enough for the one-launch inverse
  DevBuf capsel;                  // the capacitance set: scores, kept indices, vertices, frames, K
  DevBuf red;                     // reduction scratch
  DevBuf flags;                   // int32 status flags
  DevBuf scal;                    // double scalars
  DevBuf io;                      // staging for host-memory calls
  DevBuf gmres;                   // GMRES basis + Hessenberg
  DevBuf fgmres;                  // flexible GMRES: preconditioned basis Z
  DevBuf xpos;                    // x in elimination order before the product with S (FP64, FP32)
  DevBuf inner;                   // inner GMRES on the capacitance: basis and scratch
  DevBuf fwd;                     // forward Newton vectors
  DevBuf fibre;                   // double [nt][3] actuation fibres (empty: none set)
  DevBuf model;                   // int8 [nt] constitutive model per tet (valid when model_any)
  bool model_any = false;         // some tet is not Neo-Hookean
  const int8_t* model_ptr() const { return model_any ? static_cast<const int8_t*>(model.p) : nullptr; }
  DevBuf actf;                    // forward: f_ext + actuation force [3 nv]; adjoint: dL/da staging
  DevBuf vec32;                   // FP32 scratch of the mixed path
  DevBuf xsplit;                  // float2 [3 nv]: double-float pairs of the Arnoldi matvec's input (mixed)
  int* flags_host = nullptr;      // pinned
  double* scal_host = nullptr;    // pinned
  double* gs_host = nullptr;      // pinned: Gram-Schmidt coefficients of one GMRES iteration
  double* gs_inner_host = nullptr;  // pinned: the same for the inner capacitance solve, and its norms
  // captured GMRES step (one graph serves every step of a cycle: the kernels read j on the device)
  double* gs_map_host = nullptr;    // host-mapped pinned slots for the captured step's coefficients
  double* gs_map_dev = nullptr;     // its device address
  DevBuf gstep;                     // int j of the captured step
  cudaGraphExec_t step_exec = nullptr;
  std::vector<uintptr_t> step_key;  // what the captured graph depends on
  int step_launches = 0;            // kernels in one replay
  cudaEvent_t ev[8] = {};
  cudaEvent_t gs_ev[2] = {};       // GMRES: coefficients of step j landed in pinned slot j % 2

  // batched per-scene GMRES (batch scenes)
  DevBuf segt;                      // int32 tiles of the DOF range: scene [n], beg [n], end [n], t0 [n_scenes + 1]
  int n_tiles = 0;
  DevBuf bwork;                     // per-scene Krylov state (flags, Hessenberg, rotations, norms, partials)
  int* bmap_host = nullptr;         // host-mapped ints: active scenes after each step, scenes not done
  int* bmap_dev = nullptr;
  cudaEvent_t bev[4] = {};          // batch steps in flight
  cudaGraphExec_t bstep_exec = nullptr;
  std::vector<uintptr_t> bstep_key;
  int bstep_launches = 0;
  std::vector<int> last_iters;      // per-scene Krylov iterations and relative residuals of the last
  std::vector<double> last_rel;     // batched adjoint
  DevBuf bio, bio_ids, btab;        // ncpadj_adjoint_batch: union staging, ids, copy tables
  void* btab_host = nullptr;        // pinned copy tables
  size_t btab_host_bytes = 0;
};

struct Ctx {
  int device = 0;
  int sm_count = 0;
  int coop_ok = 0;
  DevBuf inv_mat, inv_work;  // workspace of ncpadj_dense_inverse
  DevBuf gemm_flags;         // status flags of ncpadj_dense_gemm
  DevBuf rec_work;           // scratch of ncpadj_dense_inverse's tensor-core blocked Gauss-Jordan
};

// looks up (and so loads) the static scratch of ncpadj_elastic_solve_noalloc on `device`, which
// must be current; called by ncpadj_ctx_create (noalloc.cu)
void noalloc_prepare(int device);

// kernels launch helpers (kernels.cu)
struct AdjointArgs;  // defined in kernels.cuh
}  // namespace ncpadj

struct ncpadj_ctx_s {
  ncpadj::Ctx c;
};
struct ncpadj_scene_s {
  ncpadj::Scene s;
  ncpadj_ctx_s* ctx = nullptr;
};
