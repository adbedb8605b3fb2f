/*
 * ncpadj -- analytical adjoint of one implicit time step of a Neo-Hookean tet mesh with
 * smoothed Signorini-Coulomb (Fischer-Burmeister) contact, on one NVIDIA GB300 (sm_103a).
 *
 * Method: "Fast and Reliable Gradients for Deformables Across Frictional Contact Regimes".
 * One call of ncpadj_adjoint_step computes, for a converged forward state,
 *   script_A^T z = dL/dq + dL/dv / h                                  (Eq. adjoint, Sec. 4.1)
 *   script_A = A - Delta A + h^2 J_c^T K_c J_c                         (Eq. differential_2)
 * with the per-tet SVD projection Jacobians of Sec. 4.3 / App. B, the per-contact smoothed
 * FB blocks of Sec. 4.2 / Eq. final_diff_contact, a Woodbury-preconditioned Krylov solve
 * (Sec. 4.4, Eq. woodbury_formula) and the gradient contractions dL/dx = z^T K_x
 * (Eq. compute_gradient, App. B.3).  Each tet may instead use the co-rotational or ARAP
 * projection of App. B.2 (ncpadj_scene_set_model); per-tet actuation (ncpadj_scene_set_fibres)
 * and bilateral bindings of vertices (ncpadj_bindings, Eq. binding) add their terms and their
 * gradients.  ncpadj_forward_step produces the converged states the adjoint needs.
 *
 * Conventions
 *  - Positions are [n_verts][3] row-major float64 (DOF 3v+r is coordinate r of vertex v).
 *  - Tets are [n_tets][4] int32, positively oriented (det[X1-X0, X2-X0, X3-X0] > 0).
 *  - Contacts are vertex-plane pairs.  frame is [n_c][3][3] row-major with rows n, t1, t2.
 *    delta_n = n . q_v - d_n,  delta_f = [t1; t2](q_v - q_prev_v) - d_f     (Eq. contact).
 *    The contact force lambda_c = (lambda_n, lambda_f1, lambda_f2) is in frame coordinates
 *    and enters the momentum equation as -h^2 J_c^T lambda_c.
 *  - Ownership: the library never frees or keeps caller pointers past a call.  Handles own
 *    only device workspace, the scene's operators and its elastic factor.
 *  - Memory: with options.memory == NCPADJ_MEM_DEVICE every array argument of
 *    ncpadj_adjoint_step is a device pointer; with NCPADJ_MEM_HOST every one is a host
 *    pointer (pinned memory recommended) and the call copies inputs in and outputs out
 *    on the given stream.  Scene descriptions are always host arrays.
 *  - Output pointers may be NULL (that output is skipped).  Non-NULL outputs are
 *    overwritten, not accumulated.
 *  - Errors: every call returns a status; nothing aborts or throws across the ABI.
 *    Invalid sizes or NULL required pointers give NCPADJ_ERR_INVALID_ARG before any
 *    launch.  ncpadj_last_error() returns a thread-local message for the last failure.
 *  - Streams: the stream is borrowed (cudaStream_t passed as void*; NULL = legacy default
 *    stream).  ncpadj_adjoint_step synchronises that stream before it returns (it reads the
 *    solver status), so it is not capturable in a CUDA graph.  On a stream other than the legacy
 *    default stream, the adjoint captures one GMRES step (Woodbury with directly inverted
 *    capacitance blocks) into a CUDA graph owned by the scene and replays it once per step; the
 *    graph is rebuilt when the scene's workspace or the contact arrays change.  On the legacy
 *    default stream the same kernels are launched one by one.
 *  - Threads: a scene's workspace is used by every call on that scene; calls on the same
 *    scene must not overlap.
 */
#ifndef NCPADJ_H
#define NCPADJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NCPADJ_OK = 0,
  NCPADJ_ERR_INVALID_ARG = 1,      /* bad size, NULL required pointer, bad option value */
  NCPADJ_ERR_CUDA = 2,             /* a CUDA runtime call failed (message in last_error) */
  NCPADJ_ERR_OOM = 3,              /* device allocation failed */
  NCPADJ_ERR_INVERTED_ELEMENT = 4, /* some tet has det F <= 0 (Neo-Hookean needs J > 0) */
  NCPADJ_ERR_NOT_CONVERGED = 5,    /* Krylov hit max_iters; outputs hold the last iterate */
  NCPADJ_ERR_NONFINITE = 6,        /* NaN/Inf met in the solve */
  NCPADJ_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up */
  NCPADJ_ERR_NOT_FACTORED = 8,     /* the scene's elastic factor is missing */
  NCPADJ_ERR_UNSUPPORTED = 9,      /* option combination not implemented */
  NCPADJ_ERR_CONTACT_DOMAIN = 10   /* a frictional contact has zero slip (no direction) */
} ncpadj_status;

enum { NCPADJ_FP64 = 0, NCPADJ_MIXED = 1, NCPADJ_TF32X3 = 2, NCPADJ_REFINED = 3 };
enum {
  NCPADJ_PRECOND_NONE = 0,
  NCPADJ_PRECOND_JACOBI = 1,   /* diag(script_A)^{-1} (Sec. 4.4, Jacobi preconditioner) */
  NCPADJ_PRECOND_ELASTIC = 2,  /* A^{-1} by the elastic factor (sparse-inverse preconditioner) */
  NCPADJ_PRECOND_WOODBURY = 3  /* (A + K_c)^{-1} by Eq. woodbury_formula (default) */
};
/* NCPADJ_SOLVER_SEMI_IMPLICIT: the stationary splitting that reuses the forward solver's structure
 * (Sec. 4.4, Eq. semi-implicit), preconditioned Richardson x^{k+1} = x^k + P^{-1}(b - B x^k); with
 * NCPADJ_PRECOND_ELASTIC (P = A) it is the paper's semi-implicit fixed-point baseline.  It
 * converges only when the spectral radius of I - P^{-1} B is below 1; a residual growing past
 * 1e6 ||b|| ends it (NOT_CONVERGED).  Offered for solver studies, never chosen by AUTO. */
enum {
  NCPADJ_SOLVER_AUTO = 0,
  NCPADJ_SOLVER_CG = 1,
  NCPADJ_SOLVER_GMRES = 2,
  NCPADJ_SOLVER_BICGSTAB = 3,
  NCPADJ_SOLVER_SEMI_IMPLICIT = 4
};
enum { NCPADJ_MEM_DEVICE = 0, NCPADJ_MEM_HOST = 1 };
/* constitutive model of a tet (App. B.2), see ncpadj_scene_set_model */
enum { NCPADJ_MODEL_NEO_HOOKEAN = 0, NCPADJ_MODEL_COROTATIONAL = 1, NCPADJ_MODEL_ARAP = 2 };

typedef struct ncpadj_ctx_s* ncpadj_ctx;     /* one per device; owns the CUDA device binding */
typedef struct ncpadj_scene_s* ncpadj_scene; /* mesh + material + h + elastic factor + workspace */

/* Library version string (static storage). */
const char* ncpadj_version(void);
/* Human-readable name of a status (static storage). */
const char* ncpadj_status_string(ncpadj_status s);
/* Message of the last failure on the calling thread ("" if none); valid until the next call. */
const char* ncpadj_last_error(void);

/* Bind a context to CUDA device `device`.  *out receives the handle.  Errors: INVALID_ARG
 * (out NULL or no such device), CUDA. */
ncpadj_status ncpadj_ctx_create(int device, ncpadj_ctx* out);
/* Destroy a context (NULL is a no-op).  Scenes created from it must be destroyed first. */
void ncpadj_ctx_destroy(ncpadj_ctx ctx);

/* Scene description: all host arrays, copied during ncpadj_scene_create.
 *   rest_pos [n_verts*3] float64, tets [n_tets*4] int32, E and nu [n_tets] float64
 *   (Young's modulus > 0, Poisson ratio in (-1, 0.5)), density > 0 (kg/m^3), h > 0 (s).
 * Lumped mass m_v = density * sum_{i containing v} V_i / 4; w_i = 2 mu_i V_i (App. B.2). */
typedef struct {
  int32_t n_verts, n_tets;
  const double* rest_pos;
  const int32_t* tets;
  const double* E;
  const double* nu;
  double density, h;
} ncpadj_scene_desc;

/* Build a scene: per-tet operators, lumped mass, the scalar elastic matrix
 * A_s = M_s + h^2 sum_i w_i B_i^T B_i (A = A_s (x) I_3, Eq. dynamics), its nested-dissection
 * Cholesky factor A_s = L L^T and the sparse inverse S = L^{-1} (Sec. 3, sparse-inverse
 * factorisation), and the fixed block pattern of script_A (Sec. 4.4, matrix assembly).
 * Errors: INVALID_ARG (sizes, indices out of range, inverted rest tet, bad material),
 * OOM, CUDA. */
ncpadj_status ncpadj_scene_create(ncpadj_ctx ctx, const ncpadj_scene_desc* desc, ncpadj_scene* out);
/* Destroy a scene (NULL is a no-op). */
void ncpadj_scene_destroy(ncpadj_scene scene);

/* A batch of independent scenes solved together (the batched adjoint).  The scene built is the
 * disjoint union of the n_scenes meshes: the vertices of mesh s are numbered after those of meshes
 * 0..s-1 (tets likewise), and every array argument of the other calls is the concatenation of
 * the per-mesh arrays in that order (ncpadj_adjoint_batch takes per-mesh arrays instead).  All
 * meshes must share h.  Each mesh's elastic factor is built independently (host threads); the
 * union's matrices are block-diagonal.  In ncpadj_adjoint_step / ncpadj_forward_step on a batch:
 *  - contacts must be grouped by mesh (non-decreasing mesh of their vertex); the contact
 *    capacitance is inverted block by block, one dense block per mesh with contacts (a mesh
 *    with more contacts than ncpadj_options.cap_block allows is solved iteratively, see there,
 *    except in the adjoint's per-mesh solve below);
 *  - the forward step gives each mesh its own line search;
 *  - the adjoint (solver AUTO or GMRES) solves every mesh by its own GMRES, as
 *    ncpadj_adjoint_batch does (stats.iterations is then the largest per-mesh count and
 *    stats.rel_residual the largest per-mesh residual); with CG or BiCGSTAB asked for by name it
 *    scales each mesh's right-hand side to unit norm and solves the union once with the tolerance
 *    rtol / sqrt(number of meshes with a nonzero seed), so every mesh's own relative residual is
 *    at most rtol.
 * Errors: as ncpadj_scene_create (the message names the failing mesh). */
ncpadj_status ncpadj_scene_create_batch(ncpadj_ctx ctx, int32_t n_scenes, const ncpadj_scene_desc* descs,
                                        ncpadj_scene* out);

/* Shells: a mesh of triangles with thickness tau and isometric bending, the 2D formulation of
 * App. B.1.  A triangle's F = D_s D_m^{-1} is 3 x 2 (D_m: the rest edges in the triangle's own
 * plane); its projection p(F) uses the thin SVD F = U diag(sigma) V^T of the same three models
 * (ncpadj_scene_set_model), with the out-of-plane rows of dP/dF equal to theta_j / sigma_j; the
 * element weight is w_i = 2 mu_i A_i tau and the lumped mass m_v = density tau sum A_i / 3.
 * Bending (Bergou et al. 2006, a quadratic model for inextensible surfaces): per interior edge e
 * with the cotangent stencil K_e of its four vertices, the energy 1/2 bend (3/(A_1+A_2))
 * |sum_a K_a x_a|^2, whose constant Hessian bend Q joins A_s (so the Woodbury preconditioner and
 * the sparse inverse include it) and script_A; the adjoint returns dL/d(bend) per mesh.
 *   rest_pos [n_verts*3] float64, tris [n_tris*3] int32 (any orientation; an edge shared by more
 *   than two triangles is an error), E and nu [n_tris], density > 0 (kg/m^3), h > 0 (s),
 *   thickness > 0 (m), bend >= 0 (N m). */
typedef struct {
  int32_t n_verts, n_tris;
  const double* rest_pos;
  const int32_t* tris;
  const double* E;
  const double* nu;
  double density, h;
  double thickness;
  double bend;
} ncpadj_shell_desc;

/* Build a scene of n_scenes >= 1 shells (a batch as in ncpadj_scene_create_batch: meshes in order,
 * shared h).  Every other call takes it like a tet scene with n_tets = the triangles; actuation
 * fibres and bindings inside elements (ncpadj_bindings.tet) are not supported on shells.  Errors:
 * INVALID_ARG (sizes, indices out of range, a degenerate rest triangle, a non-manifold edge, bad
 * material, thickness or bend), OOM, CUDA. */
ncpadj_status ncpadj_scene_create_shells(ncpadj_ctx ctx, int32_t n_scenes, const ncpadj_shell_desc* descs,
                                         ncpadj_scene* out);
/* New bending stiffness of each mesh of a shell scene (HOST array [n_scenes], each >= 0): A_s,
 * its factor and the sparse inverse are rebuilt as by ncpadj_scene_refactor (same rules).  Errors:
 * INVALID_ARG (NULL, a tet scene, a value out of range: nothing is changed), OOM, CUDA. */
ncpadj_status ncpadj_scene_set_bending(ncpadj_scene scene, const double* bend, void* stream);
/* The current bending stiffness of each mesh (HOST array [n_scenes]; 0 for tet scenes). */
ncpadj_status ncpadj_scene_get_bending(ncpadj_scene scene, double* bend);

/* New material for an existing scene (per-tet Young's modulus E > 0 and Poisson ratio nu in
 * (-1, 0.5), HOST arrays [n_tets] over the whole scene, batch meshes concatenated).  Everything that
 * depends on the material is rebuilt from the scene's kept geometry: the Lame parameters and their
 * derivatives, A_s = M_s + h^2 sum_i w_i B_i^T B_i (w_i = 2 mu_i V_i), its Cholesky factor and the
 * sparse inverse S = L^{-1} (Sec. 3, sparse-inverse factorisation; Eq. dynamics).  The mesh, the
 * step size, the fibres and the constitutive models are kept.  Work queued on `stream` is waited
 * for first (it may read the arrays being rebuilt); the call is synchronous.  Calls on the scene
 * must not overlap it.  Errors: INVALID_ARG (NULL, a value out of range: nothing is changed),
 * OOM, CUDA. */
ncpadj_status ncpadj_scene_refactor(ncpadj_scene scene, const double* E, const double* nu, void* stream);
/* The scene's current per-tet E and nu (HOST arrays [n_tets] to fill). */
ncpadj_status ncpadj_scene_get_material(ncpadj_scene scene, double* E, double* nu);

typedef struct {
  int32_t n_verts, n_tets;
  int32_t n_blocks;        /* 3x3 blocks in the pattern of script_A */
  int64_t nnz_L;           /* nonzeros of the scalar Cholesky factor */
  int64_t nnz_Linv;        /* nonzeros of its explicit inverse S */
  double ms_factor;        /* host time of ordering + factorisation + inversion (summed over meshes) */
  int32_t n_scenes;        /* meshes in the scene (1 unless built by ncpadj_scene_create_batch) */
  int32_t element_verts;   /* 4: tets, 3: triangles (ncpadj_scene_create_shells) */
  int32_t n_hinges;        /* interior edges carrying bending (shells) */
} ncpadj_scene_info;
ncpadj_status ncpadj_scene_get_info(ncpadj_scene scene, ncpadj_scene_info* out);

/* Contact set for one call (frozen: Sec. 4.2 treats J_c and the frame as fixed).
 *   vertex [n_c] int32, frame [n_c*9] float64 (rows n, t1, t2; orthonormal),
 *   d_n [n_c], d_f [n_c*2] or NULL (= 0), mu [n_c] >= 0 (mu = 0: frictionless),
 *   region [n_c] int32 in [0, n_regions) or NULL (= 0); n_regions >= 1. */
typedef struct {
  int32_t n_contacts;
  const int32_t* vertex;
  const double* frame;
  const double* d_n;
  const double* d_f;
  const double* mu;
  const int32_t* region;
  int32_t n_regions;
} ncpadj_contacts;

/* Bilateral binding constraints on single vertices (Eq. binding), for one call.  Binding b
 * attaches vertex[b] to the point target[b] through a compliant spring:
 *   delta_b = q_v - d_b,  phi_b = delta_b + E_b lambda_b = 0,  so lambda_b = -(q_v - d_b) / E_b,
 * with the compliance E_b = compliance[b] > 0 (small E_b: a stiff attachment; J_b selects the
 * vertex's three coordinates).  The forward step gains the force h^2 (q_v - d_b) / E_b in its
 * residual, script_A gains h^2 / E_b I_3 on v's diagonal block (Eq. differential_2), and the
 * adjoint returns dL/dd_b = h^2 z_v / E_b and dL/dE_b = h^2 z_v . (q_v - d_b) / E_b^2.  The
 * Woodbury preconditioner does not include them: they perturb the preconditioned operator by a
 * matrix of rank 3 n_bindings, which Krylov absorbs in at most that many extra iterations.
 *   vertex [n_bindings] int32 in [0, n_verts), target [n_bindings*3], compliance [n_bindings]:
 *   device arrays (the call must use NCPADJ_MEM_DEVICE).  Several bindings may share a vertex.
 *   tet [n_bindings] int32 in [0, n_tets) and bary [n_bindings*4] (both, or both NULL): binding b
 *   is then the point sum_a bary[b][a] x_a of the vertices of tet[b] (a point inside the tet for
 *   barycentric weights), J_b = bary_b^T (x) I_3, its blocks h^2 w_a w_c / E_b I_3 lie in the
 *   tet's own pattern, and vertex is not read. */
typedef struct {
  int32_t n_bindings;
  const int32_t* vertex;
  const double* target;
  const double* compliance;
  const int32_t* tet;
  const double* bary;
} ncpadj_bindings;

/* Converged forward state: q, q_prev [n_verts*3]; lambda [n_c*3] contact forces in frame
 * coordinates (lambda_n, lambda_f1, lambda_f2).  The tangential multiplier used in the
 * friction blocks is gamma = -lambda_f . delta_f / ||delta_f|| (signed).  bindings: the
 * call's bilateral bindings, or NULL for none (they must be the ones the forward step used). */
typedef struct {
  const double* q;
  const double* q_prev;
  const double* lambda;
  const ncpadj_bindings* bindings;
} ncpadj_state;

/* Loss seeds dL/dq and dL/dv [n_verts*3] at the end of the step (dL_dv may be NULL = 0). */
typedef struct {
  const double* dL_dq;
  const double* dL_dv;
} ncpadj_seed;

/* Gradient outputs (each nullable):
 *   dL_dq_prev, dL_dv_prev, dL_dfext, z  [n_verts*3]
 *   dL_dE, dL_dnu                        [n_tets]   (per-tet material parameters)
 *   dL_dmu                               [n_regions] (friction coefficient per region)
 *   dL_dmu_contact                       [n_c]       (per contact)
 *   dL_dact                              [n_tets]    (FP32; per-tet activation, see
 *                                                     ncpadj_scene_set_fibres)
 *   dL_dbinding_target                   [n_b*3]     (binding targets d_b)
 *   dL_dcompliance                       [n_b]       (binding compliances E_b)
 *   dL_dbend                             [n_scenes]  (bending stiffness of each shell mesh;
 *                                                     -h^2 z^T Q q, 0 for tet scenes) */
typedef struct {
  double* dL_dq_prev;
  double* dL_dv_prev;
  double* dL_dfext;
  double* dL_dE;
  double* dL_dnu;
  double* dL_dmu;
  double* dL_dmu_contact;
  double* z;
  float* dL_dact;  /* [n_tets] activation gradient; requires the scene's fibres (see below) */
  double* dL_dbinding_target;  /* [n_b*3]; requires state.bindings */
  double* dL_dcompliance;      /* [n_b];   requires state.bindings */
  double* dL_dbend;            /* [n_scenes] */
} ncpadj_grads;

/* Solver options; fill with ncpadj_options_default first.
 *   eps        smoothing of FB_eps(x, y) = x + y - sqrt(x^2 + y^2 + 2 eps^2); must equal the
 *              forward pass's (App. A.2).  Default 1e-4.
 *   rtol       stop at ||b - script_A^T z|| <= rtol ||b||.  Default 1e-8 (Sec. 5).
 *   max_iters  Krylov iteration cap (default 2000); gmres_restart m (default 64).
 *   precision  NCPADJ_FP64 (default) or NCPADJ_MIXED: FP32 matrix values (per-tet SVD Jacobians in
 *              FP32), FP32 matvec and preconditioner apply, FP64 vectors, dot products,
 *              Gram-Schmidt and Hessenberg; contact blocks always from FP64 state.
 *   precond    NCPADJ_PRECOND_* (default WOODBURY); solver NCPADJ_SOLVER_* (default AUTO:
 *              CG when every mu is 0, else GMRES, Sec. 4.4; NCPADJ_SOLVER_BICGSTAB on request:
 *              right-preconditioned BiCGSTAB, no restart, at least 7 vectors of workspace; an
 *              inner iterative capacitance solve makes the preconditioner vary, and then GMRES
 *              (flexible) is used whatever is asked); memory NCPADJ_MEM_*.
 *   cap_precision  inversion of the contact capacitance I + h^2 K^T D: NCPADJ_FP64 (default),
 *              NCPADJ_MIXED (inverted by Gauss-Jordan and applied in FP32; it only preconditions,
 *              so the result keeps the solve's precision and tolerance), NCPADJ_TF32X3 (FP32,
 *              inverted by the blocked Gauss-Jordan elimination of ncpadj_dense_inverse whose
 *              rank-64 updates run on the tensor cores; pivoting only inside its 64 x 64
 *              diagonal blocks) or NCPADJ_REFINED (the TF32X3 inverse X, and every capacitance
 *              solve refined once against the FP64 capacitance C: x = X y, x += X (y - C x), an
 *              FP64-accurate solve while ||I - C X|| is small; directly inverted blocks only).
 *   cap_block  most contacts per directly inverted capacitance block (0 = default = 2730 with an
 *              FP32 capacitance, 1365 with FP64; at most 5461 resp. 1365).  A scene with
 *              more contacts has its capacitance solved iteratively (Sec. 4.4): an inner
 *              right-preconditioned GMRES to relative residual 1e-6 applies the capacitance
 *              without forming it (a scatter and a gather along the contacts' elimination-tree
 *              paths per product), preconditioned by the exact inverses of contiguous, nearly
 *              equal groups of its contacts in the given order; the outer solve becomes flexible
 *              GMRES (the preconditioner varies).  Order the contacts spatially (e.g. by plane,
 *              then by position) so that groups are compact.
 *   cap_drop   contacts whose rows of the capacitance stand within this of the identity are left
 *              out of it: contact c is dropped when h^2 |K_c|_F (A^{-1})_{v_c v_c} <= cap_drop
 *              (default 1e-2; 0 keeps every contact).  A separating contact, whose blocks are
 *              ~eps^2/delta_n^2, scores far below that, an active one far above.  The Woodbury
 *              preconditioner is then exact for the kept contacts; the dropped ones stay in the
 *              matrix, so the result keeps its tolerance.  stats.capacitance_dim counts the kept
 *              rows. */
typedef struct {
  double eps, rtol;
  int32_t max_iters, gmres_restart;
  int32_t precision, precond, solver, memory;
  int32_t cap_precision;
  int32_t cap_block;
  double cap_drop;
} ncpadj_options;
void ncpadj_options_default(ncpadj_options* opt);

/* Per-call statistics (nullable).  Times are CUDA-event times of the stages on the stream. */
typedef struct {
  int32_t iterations;       /* Krylov iterations */
  int32_t solver_used;      /* NCPADJ_SOLVER_CG, _GMRES, _BICGSTAB or _SEMI_IMPLICIT */
  int32_t n_contacts;
  int32_t capacitance_dim;  /* dimension of the dense contact-space system (0 if none) */
  double rel_residual;      /* final ||b - script_A^T z|| / ||b|| (recomputed explicitly) */
  float ms_total, ms_assemble, ms_setup, ms_krylov, ms_contract;
  float ms_cap_inverse;     /* the capacitance inversion kernel alone (0 if not run) */
  int64_t kernel_launches;  /* kernels this call enqueued */
  int32_t capacitance_blocks;  /* capacitance blocks inverted directly (0 if none) */
  int32_t inner_iterations;    /* iterations of the inner capacitance solves (0 if none) */
} ncpadj_stats;

/* One adjoint step: assemble script_A^T at the given converged state, solve for z and
 * contract the gradients.  Errors: INVALID_ARG (including a contact or binding vertex out of
 * range, a compliance that is not positive, bindings with NCPADJ_MEM_HOST, binding gradients
 * without bindings), INVERTED_ELEMENT, CONTACT_DOMAIN, NOT_CONVERGED (outputs hold the last
 * iterate's gradients, stats the residual), NONFINITE, TIMEOUT, OOM, CUDA. */
ncpadj_status ncpadj_adjoint_step(ncpadj_ctx ctx, ncpadj_scene scene, const ncpadj_contacts* contacts,
                                  const ncpadj_state* state, const ncpadj_seed* seed,
                                  const ncpadj_options* opt, ncpadj_grads* grads,
                                  ncpadj_stats* stats, void* stream);

/* Batched adjoint: one adjoint step of every mesh of a batch scene (ncpadj_scene_create_batch) in
 * one call -- the many-scene workload of the paper's batched differentiable simulation (Sec. 5),
 * with the Krylov solve of Sec. 4.4 (Eq. adjoint, Eq. woodbury_formula) run scene by scene.
 *   n_scenes     the batch's number of meshes (else INVALID_ARG).
 *   contacts     [n_scenes] or NULL (no contacts anywhere); states, seeds [n_scenes] (required);
 *   grads, stats [n_scenes] or NULL.  Entry s describes mesh s exactly as the arguments of
 *                ncpadj_adjoint_step would describe that mesh alone: vertex ids in [0, its n_verts),
 *                regions in [0, its n_regions), every array sized for that mesh, NULL outputs
 *                skipped.  All arrays are device pointers, or all host pointers with
 *                options.memory = NCPADJ_MEM_HOST.
 * Every mesh runs its own right-preconditioned flexible GMRES: its own inner products, Hessenberg
 * matrix, restarts and stopping test ||b_s - script_A_s^T z_s|| <= rtol ||b_s||.  The meshes share
 * every kernel launch of a Krylov step; a mesh that has converged drops out of the later launches
 * (their kernels skip its rows), so a call costs about the sum of the meshes' own iterations,
 * not their number times the slowest one's.  Off the legacy default stream each step is one replay
 * of a captured CUDA graph owned by the scene.  Capacitance blocks above the direct inverse's size
 * are split into directly inverted groups (no inner solve).
 * stats[s].iterations, .rel_residual and .n_contacts are mesh s's own; the times, kernel_launches
 * and capacitance fields describe the whole call.
 * Not supported here: bindings (states[s].bindings must be NULL) and solvers other than AUTO or
 * GMRES (UNSUPPORTED).  Synchronises the stream.
 * Errors: as ncpadj_adjoint_step (a contact vertex or region outside its own mesh's range is
 * INVALID_ARG); NOT_CONVERGED when some mesh stopped above rtol -- every output is still written
 * and that mesh's stats entry shows its residual. */
ncpadj_status ncpadj_adjoint_batch(ncpadj_ctx ctx, ncpadj_scene batch, int32_t n_scenes,
                                   const ncpadj_contacts* contacts, const ncpadj_state* states,
                                   const ncpadj_seed* seeds, const ncpadj_options* opt,
                                   ncpadj_grads* grads, ncpadj_stats* stats, void* stream);

/* y = A^{-1} x for the elastic matrix A = M + h^2 sum_i w_i G_i^T G_i of the scene (Eq. dynamics),
 * applied through the scene's sparse-inverse factorisation A^{-1} = P^T S^T S P (Sec. 3).
 * x, y: device arrays [n_verts*3] (not aliased).  Uses the scene's workspace (allocated on first
 * use).  Errors: INVALID_ARG, OOM, CUDA. */
ncpadj_status ncpadj_elastic_solve(ncpadj_ctx ctx, ncpadj_scene scene, const double* x, double* y, void* stream);

/* The same product as ncpadj_elastic_solve in the mixed precision of the preconditioner
 * (ncpadj_options.precision = NCPADJ_MIXED): FP32 values of S = L^{-1} and FP32 intermediates,
 * FP64 x and y.  Same arguments and errors. */
ncpadj_status ncpadj_elastic_solve_mixed(ncpadj_ctx ctx, ncpadj_scene scene, const double* x, double* y,
                                         void* stream);

/* Per-tet actuation (the paper's muscle-driven soft robots describe their actuators only in words;
 * this is the reading used here): tet i carries an activation a_i (Pa, FP32) and a fixed unit fibre
 * direction d_i in the rest frame, adding the constant first Piola stress a_i d_i d_i^T.  Its nodal
 * force f_act = - sum_i V_i G_i^T vec(a_i d_i d_i^T) does not depend on q, so it joins f_ext in the
 * forward step (ncpadj_forward_input.act) and leaves the adjoint matrix unchanged; the adjoint
 * returns dL/da_i = h^2 z^T df_act/da_i = -h^2 V_i d_i^T Z_i d_i with Z_i = unvec(G_i z)
 * (ncpadj_grads.dL_dact).
 * fibre: HOST array [n_tets*3] of unit vectors (copied; replaces earlier fibres of the scene).
 * Errors: INVALID_ARG (NULL, or a fibre whose length is not 1 within 1e-6), OOM, CUDA. */
ncpadj_status ncpadj_scene_set_fibres(ncpadj_scene scene, const double* fibre);

/* Constitutive model per tet.  The three isotropic models of App. B.2 share the SVD projection
 * Jacobian of Sec. 4.3 and differ only in the projection theta(sigma) of the singular values:
 *   NCPADJ_MODEL_NEO_HOOKEAN (default): zeta = mu/2 (I_1 - log I_3 - 3) + lambda/8 (log I_3)^2;
 *   NCPADJ_MODEL_COROTATIONAL: zeta = mu ||theta - 1||^2 + lambda/2 (sum_i (theta_i - 1))^2, whose
 *     projection is linear: theta - 1 = W (sigma - 1) with the constant
 *     W = I/2 - lambda / (2 (4 mu + 3 lambda)) 1 1^T;
 *   NCPADJ_MODEL_ARAP: theta = 1 (p(F) is the rotation of F); lambda plays no part and mu only
 *     sets the weight w = 2 mu (the stretch stiffness).
 * Every model weights tet i by w_i = 2 mu_i V_i, so the elastic factor does not change.  Every
 * model rejects det F <= 0 (INVERTED_ELEMENT).  The forward and adjoint steps and the E, nu
 * gradients follow the model of each tet.
 * model: HOST array [n_tets] of NCPADJ_MODEL_* (copied), or NULL to make every tet Neo-Hookean.
 * Errors: INVALID_ARG (NULL scene, a value that is no NCPADJ_MODEL_*), OOM, CUDA. */
ncpadj_status ncpadj_scene_set_model(ncpadj_scene scene, const int32_t* model);

/* Launch shape of the product with A^{-1} = P^T S^T S P (the sparse-inverse preconditioner of
 * Sec. 3, GPU acceleration via sparse-inverse factorization; the paper fixes no launch shape): the
 * rows of S and S^T are cut into chunks of at most `entries` nonzeros, one warp per chunk with
 * entries / 32 values in flight per lane.  128, 256 (the default) or 512; the best depends on the
 * scene's factor and is found by timing (paper_2603_16478_gb300.autotune).  Results agree to
 * rounding (the chunks' partial sums are added in a different grouping).  Takes effect from the
 * next call on the scene; a refactor keeps it.
 * Errors: INVALID_ARG (NULL scene, another size), OOM, CUDA. */
ncpadj_status ncpadj_scene_set_chunk(ncpadj_scene scene, int32_t entries);

/* Cinv = C^{-1} for a dense row-major n x n matrix, by the blocked Gauss-Jordan elimination with
 * partial pivoting that inverts the contact capacitance I + h^2 K D of the Woodbury
 * preconditioner (Sec. 4.4); exposed so that the inversion can be used and checked on its own.
 * C, Cinv: device arrays [n*n] (not aliased; C is not modified).  precision NCPADJ_FP64 computes
 * in FP64; NCPADJ_MIXED rounds C to FP32 and computes in FP32 (the result is returned as double);
 * NCPADJ_TF32X3 rounds C to FP32 and inverts it by blocked Gauss-Jordan elimination, 64 columns
 * per step, in one persistent cooperative launch: each step's 64 x 64 diagonal block is inverted
 * with pivoting among its own rows, and the rank-64 update of the whole matrix runs on the tensor
 * cores (tcgen05.mma kind::tf32 with the 3xTF32 split, about FP32 accuracy).  There is no pivoting
 * across blocks: every diagonal block met along the way must be invertible (else NONFINITE).
 * 1 <= n <= 16384 (FP64: n <= 4096, else UNSUPPORTED).  Synchronises the stream (it reads the
 * pivot status).  Uses workspace owned by
 * the context (allocated on first use, grown as needed).
 * Errors: INVALID_ARG, NONFINITE (a zero pivot: C is singular in the working precision),
 * TIMEOUT, UNSUPPORTED (the cooperative launch was refused), OOM, CUDA. */
ncpadj_status ncpadj_dense_inverse(ncpadj_ctx ctx, int32_t n, const double* C, double* Cinv, int32_t precision,
                                   void* stream);

/* C = alpha A B + beta C on the fifth-generation tensor cores (tcgen05.mma, kind::tf32, FP32
 * accumulation in tensor memory), the dense product the capacitance inverse of the Woodbury
 * preconditioner (Sec. 4.4) is built from, exposed so that it can be used and checked on its own.
 * A [M][K], B [K][N], C [M][N]: row-major FP32 DEVICE arrays with leading dimensions lda >= K,
 * ldb >= N, ldc >= N (elements); C must not overlap A or B.  split = 1 splits every operand into a
 * TF32 head and tail and adds the three leading products (about FP32 accuracy: relative error of a
 * product ~1e-6 of sum |a_ik b_kj|); split = 0 rounds the operands to TF32 (~1e-3).  beta = 0 does
 * not read C.  Synchronises the stream (it reads the kernel's status).
 * Errors: INVALID_ARG, TIMEOUT (a wait of the kernel gave up), OOM, CUDA. */
ncpadj_status ncpadj_dense_gemm(ncpadj_ctx ctx, int32_t M, int32_t N, int32_t K, float alpha, const float* A,
                                int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                                int32_t split, void* stream);

/* Variant of ncpadj_elastic_solve that allocates nothing (the paper has no counterpart).
 * For callers that cannot have device memory allocated while they run -- programs whose device
 * memory is reserved up front by their own pool, or loops with hard latency limits where a
 * cudaMalloc is not acceptable.  Same arguments and result as ncpadj_elastic_solve; the
 * intermediate vectors live in a static device array sized for at most 262,144 vertices
 * (12 MiB, held by every GPU on which a context is created, until the process exits).
 *  - Scenes with more vertices are rejected with NCPADJ_ERR_INVALID_ARG.
 *  - The call makes no cudaMalloc or cudaFree.  ncpadj_ctx_create looks up the array's device
 *    address (cudaGetSymbolAddress), which makes CUDA load it: the array is allocated when the
 *    context is created, never during this call.
 *  - Every call shares the one array: calls that overlap on the GPU (other streams, other
 *    threads) race with each other.  Each call clears the array before use.
 * Errors: INVALID_ARG, CUDA. */
ncpadj_status ncpadj_elastic_solve_noalloc(ncpadj_ctx ctx, ncpadj_scene scene, const double* x, double* y,
                                           void* stream);

/* ---- forward step -------------------------------------------------------------------------
 * The converged state that ncpadj_adjoint_step differentiates.  One implicit Euler step of
 * Eq. (dynamics): q minimises the incremental potential of Eq. (implicit) with the projective
 * Neo-Hookean force of Eq. (internal) and the smoothed-FB contact conditions of Eq. (contact).
 * Solved by Newton's method in q alone: the multipliers are eliminated by the exact local
 * solution of the contact equations (lambda_n = eps^2 / delta_n, and along -t = -delta_f/||delta_f||
 * the friction magnitude gamma = mu lambda_n - eps^2/||delta_f||), so the Newton matrix is script_A
 * itself, solved by the same Woodbury-preconditioned Krylov method.  A backtracking line search
 * keeps every contact inside that local-solve domain and does not let the slip of a contact
 * carrying friction turn by more than 60 degrees in one step.
 *   q_prev, v_prev [n_verts*3] (v_prev may be NULL = 0); f_ext [n_verts*3] forces besides
 *   gravity or NULL; gravity: acceleration vector (m/s^2).
 * All arrays are device pointers (options.memory must be NCPADJ_MEM_DEVICE). */
typedef struct {
  const double* q_prev;
  const double* v_prev;
  const double* f_ext;
  double gravity[3];
  const float* act;  /* [n_tets] activations (Pa) or NULL; requires the scene's fibres */
  const ncpadj_bindings* bindings;  /* bilateral bindings of the step, or NULL */
} ncpadj_forward_input;

typedef struct {
  int32_t newton_iters, krylov_iters;
  double residual;  /* ||R_q|| / (h^2 ||M g||) at the returned state */
  float ms_total;
} ncpadj_forward_stats;

/* Outputs: q_out [n_verts*3], lambda_out [n_c*3] (frame coordinates, required if n_c > 0).
 * Stops when ||R_q|| <= newton_tol h^2 ||M g|| or when no step decreases ||R_q|| any more.
 * Errors: INVALID_ARG, UNSUPPORTED, CONTACT_DOMAIN (no start point inside the local-solve
 * domain), INVERTED_ELEMENT, NOT_CONVERGED (residual above 1e3 newton_tol), NONFINITE, OOM, CUDA. */
ncpadj_status ncpadj_forward_step(ncpadj_ctx ctx, ncpadj_scene scene, const ncpadj_contacts* contacts,
                                  const ncpadj_forward_input* input, const ncpadj_options* opt, double newton_tol,
                                  int32_t max_newton, double* q_out, double* lambda_out, ncpadj_forward_stats* stats,
                                  void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NCPADJ_H */
