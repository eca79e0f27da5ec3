/*
 * fem.h - C ABI of the GB300 (sm_103a) partial-assembly finite-element library.
 *
 * The library computes the matrix-free (partially assembled) action y = A x of
 * the high-order H1 mass and diffusion operators on unstructured hexahedral
 * Q_p meshes by sum factorization, the assembled diagonal, the load vector,
 * the Jacobi-preconditioned CG solve built on the action (FP64, double-float,
 * or FP32 inner iterations inside FP64 iterative refinement), batched
 * applies/solves over many independent problems, and the compliance gradient
 * with respect to a per-element coefficient. Beside these: quadrilateral (2D)
 * meshes, curved (order-k nodal) geometry, the convection and linear
 * elasticity forms, and a p-multigrid preconditioner with flexible CG.
 *
 * The operator follows the decomposition A = P^T G^T B^T D B G P of the paper
 * (Sec. 4.3 "Operator Decomposition"; P = I on one GPU): G is the element
 * restriction (L-vector -> E-vector gather, its transpose an atomic-free
 * scatter-add through an inverse map), B the sum-factorized basis evaluator
 * (Sec. 4.4, B_ki as a product of 1D factors), D the point-wise quadrature
 * data stored by the setup phase (Sec. 4.4, "partial assembly operates at the
 * Q-vector level ... leaves only the D operator to store").
 *
 * Conventions (all entry points):
 *  - Every call returns fem_status; FEM_OK == 0. No call aborts, throws or
 *    traps on the device. fem_last_error() returns a thread-local message for
 *    the last failing call of the calling thread.
 *  - Handles (fem_mesh, fem_space, fem_form, fem_batch) are opaque and owned
 *    by the library; destroy them with the matching *_destroy call. A space
 *    must outlive the forms built on it; a mesh must outlive its spaces.
 *  - Vectors passed as `void*` / `double*` device pointers are caller-owned
 *    CUDA device memory (e.g. torch tensor data pointers), contiguous, and
 *    of the dtype named by the call. Host pointers are named `*_host`.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *    asynchronous on that stream unless documented otherwise.
 *  - Output vectors must not alias input vectors.
 *  - L-vector ordering: global DOF numbering of Sec. 3.4 ("Finite Element
 *    Spaces"): vertices (vertex id), then edges, then faces, then element
 *    interiors. Edges/faces are numbered by first appearance scanning elements
 *    in order and, inside an element, the local edge order
 *    (0,1),(1,2),(3,2),(0,3),(4,5),(5,6),(7,6),(4,7),(0,4),(1,5),(2,6),(3,7)
 *    and face order z=0,y=0,x=1,y=1,x=0,z=1. Edge DOFs run from the lower to
 *    the higher global vertex; face DOFs are listed row by row in the frame at
 *    the face's lowest global vertex, first axis toward the lower-numbered of
 *    its two face neighbours. Interiors: lexicographic, x fastest.
 *  - Reference cell [0,1]^3; local hexahedron vertex order: bottom face 0-1-2-3
 *    counter-clockwise seen from above, top face 4-5-6-7 (VTK order). The map
 *    is trilinear in the 8 vertices (Sec. 3.1, Eq. mesh_eq_x with vertex
 *    coordinates). Basis: nodal Lagrange at Gauss-Lobatto points (Sec. 3.3);
 *    quadrature: q1d-point Gauss-Legendre per direction.
 */
#ifndef FEM_H
#define FEM_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fem_status;
enum {
  FEM_OK = 0,
  FEM_EINVAL = 1,        /* bad argument, size or mesh connectivity */
  FEM_ENOMEM = 2,        /* device or host allocation failed */
  FEM_EINVERTED = 3,     /* setup found det J <= 0 at a quadrature point */
  FEM_ENOCONV = 4,       /* solver hit maxit before the tolerance */
  FEM_EBREAKDOWN = 5,    /* CG breakdown: p^T A p <= 0 or a non-finite scalar */
  FEM_ECUDA = 6,         /* a CUDA runtime call or kernel launch failed */
  FEM_EUNSUPPORTED = 7   /* (p, q1d) or size outside the compiled set */
};

enum { FEM_MASS = 0, FEM_DIFFUSION = 1, FEM_CONVECTION = 2, FEM_ELASTICITY = 3 };  /* bilinear form kind */
/* Vector / compute type. FEM_DF64: float64 vectors, element arithmetic in
 * double-float (pairs of floats, 48-bit significand, on the FP32 pipe) with a
 * double-float copy of D made on first use; the operator agrees with the FP64
 * one to about 1e-13 relative (values must stay within about 1e+-30). */
enum { FEM_F64 = 0, FEM_F32 = 1, FEM_DF64 = 2 };
/* Solve precision: FP64 CG; FP32 inner CG restarted inside FP64 iterative
 * refinement; FP64 CG whose operator applies run in double-float
 * (FEM_DF64); FP32 CG with FP64 reliable updates (the FP32 increment is
 * folded into the FP64 solution and the residual replaced by the FP64 true
 * residual whenever it has dropped by inner_rtol, without restarting the
 * search direction). */
enum { FEM_SOLVE_F64 = 0, FEM_SOLVE_MIXED = 1, FEM_SOLVE_DF64 = 2, FEM_SOLVE_MIXED_RU = 3 };
/* Preconditioner of fem_solve: Jacobi (assembled diagonal, Sec. 5.2) or none
 * (plain CG, the iteration of the paper's Example 1 timings, Sec. 5.3). */
enum { FEM_PC_JACOBI = 0, FEM_PC_NONE = 1 };

typedef struct fem_mesh fem_mesh;
typedef struct fem_space fem_space;
typedef struct fem_form fem_form;
typedef struct fem_batch fem_batch;

/* Library version string and thread-local description of the last error. */
const char* fem_version(void);
const char* fem_last_error(void);

/* Orders p and 1D quadrature sizes q1d compiled into this build.
 * fem_supported(p, q1d) returns 1 if the pair has kernels, else 0. */
int fem_supported(int p, int q1d);

/* ---- mesh (Sec. 3.1 "Conforming Meshes": vertices + element vertex tuples) --
 * coords_host: [nv][3] float64 vertex coordinates; hex_host: [ne][8] int32
 * vertex indices in the local order above. Both are copied (host + device);
 * the caller keeps ownership of its arrays. Errors: FEM_EINVAL if nv or ne is
 * not positive, an index is out of range, an element repeats a vertex or a
 * vertex is referenced by no element. */
fem_status fem_mesh_create(const double* coords_host, int64_t nv,
                           const int32_t* hex_host, int64_t ne, fem_mesh** out);
/* Quadrilateral (2D) mesh, the d = 2 case of the same definitions:
 * coords_host [nv][2] float64; quad_host [ne][4] int32, local vertex order
 * 0:(0,0) 1:(1,0) 2:(1,1) 3:(0,1) (counter-clockwise on [0,1]^2, bilinear
 * map). Everything built on it takes the 2D shapes stated below ((p+1)^2
 * local DOFs, q1d^2 points, [..][2] coordinates); batches may mix
 * quadrilateral and hexahedral problems. Same ownership and errors as
 * fem_mesh_create. */
fem_status fem_mesh2d_create(const double* coords_host, int64_t nv,
                             const int32_t* quad_host, int64_t ne, fem_mesh** out);
/* High-order (curved) geometry, Sec. 3.1 "nodes": element e is mapped by
 * x(xhat) = sum_i X_{e,i} w_i(xhat) with the (k+1)^dim order-k GLL Lagrange
 * functions w_i (lexicographic, x fastest, in the element's local vertex
 * frame). nodes_host: [ne][(k+1)^3][3] float64 on a hexahedral mesh,
 * [ne][(k+1)^2][2] on a quadrilateral one, copied; 1 <= k <= 8, or k = 0 to
 * return to the multilinear vertex map. Forms created afterwards use it in
 * their setup (D), load vector and coordinates (quadrature points and DOFs);
 * an existing form picks it up at its next fem_form_set_coef. The vertex
 * coordinates still define the topology. Errors: FEM_EINVAL (order,
 * non-finite coordinates). */
fem_status fem_mesh_set_nodes(fem_mesh* mesh, int k, const double* nodes_host);
void fem_mesh_destroy(fem_mesh* mesh);

/* ---- H1 space of order p (Sec. 3.4 "Finite Element Spaces") ----------------
 * Builds the global numbering, the element->DOF table e2l [ne][(p+1)^3]
 * (lexicographic local order, x fastest), its inverse (CSR, entries sorted by
 * element then local index: the fixed summation order of the scatter) and the
 * boundary DOFs (DOFs on faces with exactly one adjacent element). On a 2D
 * mesh: vertices, then edges by first appearance (local edges (0,1), (1,2),
 * (3,2), (0,3), DOFs from the lower to the higher global vertex), then
 * interiors; e2l [ne][(p+1)^2]; boundary = edges with one element. Host-side
 * setup, synchronous. Errors: FEM_EINVAL (p < 1), FEM_EUNSUPPORTED (p > 8 or
 * ne (p+1)^3 >= 2^31). */
fem_status fem_space_create(const fem_mesh* mesh, int p, fem_space** out);
void fem_space_destroy(fem_space* space);
fem_status fem_space_info(const fem_space* space, int64_t* ndof, int64_t* nbdr,
                          int64_t* ne, int* p);
/* Boundary DOF ids, ascending: out_host [nbdr] int32. */
fem_status fem_space_boundary_dofs(const fem_space* space, int32_t* out_host);
/* The element->DOF table: out_host [ne][(p+1)^3] int32. */
fem_status fem_space_element_dofs(const fem_space* space, int32_t* out_host);
/* Physical location of every DOF (the trilinear map of its first element at
 * the GLL node): out [ndof][3] float64 device ([ndof][2] in 2D).
 * Asynchronous on stream. */
fem_status fem_space_dof_coords(const fem_space* space, double* out, void* stream);

/* ---- partial-assembly setup (Sec. 4.3: setup phase "evaluates and stores D")
 * kind = FEM_DIFFUSION stores, per element e and quadrature point q,
 *   D_q = coef_e w_q det J_q J_q^-1 J_q^-T  (6 symmetric components
 *   00,01,02,11,12,22; the 3D form of the diffusion setup listing of
 *   Sec. 5.3, which stores alpha W adj(J) adj(J)^T / det J in 2D);
 * kind = FEM_MASS stores D_q = coef_e w_q det J_q (Sec. 4.4, (D_E)_kk).
 * coef: device float64 [ne] per-element coefficient, or NULL for 1.
 * Layout in HBM: [ne][q1d^3][6] (diffusion, the six components of a point
 * contiguous) or [ne][q1d^3] (mass), float64, point index lexicographic
 * (x fastest). 2D: [ne][q1d^2][3] (components 00, 01, 11) or [ne][q1d^2].
 * Synchronises `stream` to read the
 * det J check. Errors: FEM_EINVERTED if any det J <= 0, FEM_EUNSUPPORTED if
 * (p, q1d) is not compiled. */
fem_status fem_form_create(const fem_space* space, int kind, int q1d,
                           const double* coef, void* stream, fem_form** out);
void fem_form_destroy(fem_form* form);
/* Convection form (beta . grad u, v) (Sec. 5.3 lists convection among the
 * partially assembled integrators): PA stores, per element and quadrature
 * point, D_q = coef_e w_q det J_q J_q^-1 beta_q = coef_e w_q adj(J_q) beta_q
 * (3 components, point-major [ne][q1d^3][3]); the apply runs the forward
 * gradient stages of the diffusion operator and the backward stages of the
 * mass operator: y = B^T (D . Ghat) x. beta_q: device float64
 * [ne][q1d^3][3], the physical velocity at the form's quadrature points
 * (fem_qpoint_coords gives their positions), copied; coef as for
 * fem_form_create. The operator is not symmetric: fem_assemble_diagonal,
 * fem_solve, fem_mg_create and fem_batch_create reject it. Hexahedral
 * meshes only (FEM_EUNSUPPORTED on 2D). */
fem_status fem_form_create_convection(const fem_space* space, int q1d, const double* beta_q,
                                      const double* coef, void* stream, fem_form** out);
/* Replace the velocity of a convection form (recomputes D). */
fem_status fem_form_set_velocity(fem_form* form, const double* beta_q, void* stream);
/* Linear elasticity a(u, v) = int lambda (div u)(div v) + 2 mu eps(u):eps(v)
 * on the vector H1 space of three components (Sec. 5.3 lists elasticity
 * among MFEM's integrators; the paper gives no elasticity kernel, so the
 * operator is written out from this definition). Vectors of an elasticity
 * form hold 3 * ndof entries, component-major ("by nodes"): component c of
 * global DOF i at c * ndof + i; essential DOF ids, the diagonal, the
 * solution and the load vector use the same numbering. PA stores, per
 * element and quadrature point, 12 float64 values [ne][q1d^3][12]:
 * J^-1 (row-major, entry 3 s + r = d xhat_s / d x_r), w det J lambda_e,
 * w det J mu_e and a zero pad. The apply computes, at every point, the
 * physical gradient H = Ghat J^-1 of the three components, the scaled
 * stress S = w det J (lambda tr(H) I + mu (H + H^T)) and F = S J^-T, then
 * runs the backward gradient stages of the diffusion operator on each
 * component of F. Its E-vector is [3][ne][(p+1)^3].
 * lambda, mu: device float64 [ne], per-element Lame coefficients, required.
 * Hexahedral meshes only; fem_compliance_grad and fem_batch_create reject
 * the form (FEM_EINVAL); fem_mg_create builds a vector hierarchy. fem_rhs takes fq
 * [3][ne][q1d^3] (the three body-force components). */
fem_status fem_form_create_elasticity(const fem_space* space, int q1d, const double* lambda,
                                      const double* mu, void* stream, fem_form** out);
/* Replace the Lame coefficients of an elasticity form (recomputes D). */
fem_status fem_form_set_lame(fem_form* form, const double* lambda, const double* mu, void* stream);
/* Replace the per-element coefficient (recomputes D). Elasticity forms take
 * fem_form_set_lame instead (FEM_EINVAL). */
fem_status fem_form_set_coef(fem_form* form, const double* coef, void* stream);
/* Essential DOF list (device int32 [n], any order, no duplicates needed):
 * defines the constrained operator A_c = (I-E) A (I-E) + E (reading of the
 * "further modifications" of FormLinearSystem, Sec. 5.1). */
fem_status fem_form_set_essential(fem_form* form, const int32_t* ess, int64_t n,
                                  void* stream);

/* ---- operator action (Sec. 4.3 apply phase; Sec. 4.4 sum factorization) ----
 * y = A x (overwrite; MFEM's AddMultPA adds, this call does not).
 * dtype FEM_F64: x, y float64, D float64 (the FP64 path).
 * dtype FEM_F32: x, y float32 with a float32 copy of D made on first use.
 * dtype FEM_DF64: x, y float64, element arithmetic in double-float.
 * constrained != 0 applies A_c (needs fem_form_set_essential).
 * Runs the element kernel (gather, B/G contractions, D, B^T/G^T) into the
 * form's E-vector scratch and the inverse-map scatter into y. */
fem_status fem_apply(const fem_form* form, int dtype, const void* x, void* y,
                     int constrained, void* stream);
/* The two halves of fem_apply with a caller-provided E-vector
 * ye [ne][(p+1)^3] ([3][ne][(p+1)^3] for elasticity) of the vector dtype
 * (float64 for FEM_DF64): element kernel, then scatter. */
fem_status fem_apply_element(const fem_form* form, int dtype, const void* x,
                             void* ye, void* stream);
fem_status fem_scatter(const fem_form* form, int dtype, const void* ye, void* y,
                       void* stream);

/* y = A x in FP64 (unconstrained), allocating nothing: the paper has no
 * counterpart; this entry point exists for callers that cannot let the
 * library allocate device memory when they call it and cannot lend it a
 * scratch buffer -- e.g. an application whose own pool has reserved nearly
 * all GPU memory, or a latency-critical loop where a cudaMalloc (which can
 * synchronise the device and can fail) is not acceptable.
 * Which fem_apply calls allocate: a constrained call (its zeroed-input work
 * vector, on first use or growth) and the first FP32 or double-float call
 * on a form (the form's converted copy of D). An unconstrained FP64
 * fem_apply reuses the E-vector buffer allocated when the form was created
 * and allocates nothing either; this entry point guarantees that by
 * construction and does not touch the form's E-vector buffer.
 * The E-vector scratch is a fixed library-owned device array of 4,194,304
 * doubles (32 MiB), held on every GPU that loads the library until the
 * process exits, in addition to every form's own E-vector buffer.
 * Limit: vdim * ne * nd <= 4,194,304 entries, with nd = (p+1)^3 on a
 * hexahedral mesh and (p+1)^2 on a quadrilateral one, and vdim = 3 for
 * elasticity (1 otherwise), else FEM_EINVAL (use fem_apply).
 * x, y: device float64 [vdim * ndof], caller-owned, not aliased.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress with that device current) and caches it for the
 * process: the cached address belongs to the device's primary context, so
 * it is stale after a cudaDeviceReset or under another context on that
 * device. Make that first call before any stream capture. Every call
 * shares the one array: calls that overlap on the GPU (other streams or
 * threads) race. The element kernel rewrites every scratch entry the
 * scatter reads, so nothing is cleared. */
fem_status fem_apply_noalloc(const fem_form* form, const double* x, double* y,
                             void* stream);

/* ---- assembled diagonal (needed for Jacobi: PA has no matrix entries,
 * Sec. 4.4 and Sec. 5.2) ----------------------------------------------------
 * diag_i = sum_e sum_q sum_ab D_ab(q) dphi_i/dxhat_a dphi_i/dxhat_b
 * (diffusion) or sum_e sum_q D(q) phi_i(q)^2 (mass); float64 device [ndof].
 * Elasticity: [3 * ndof]; component c uses the symmetric 3x3 matrix
 * w det J ((lambda + mu) a_c a_c^T + mu J^-1 J^-T), a_c = column c of J^-1,
 * in place of D (the (c, c) block's diagonal); needs ne * q1d^3 * 6
 * float64 of temporary device memory.
 * constrained != 0 sets diag = 1 on essential DOFs. */
fem_status fem_assemble_diagonal(const fem_form* form, double* diag,
                                 int constrained, void* stream);

/* ---- load vector (Sec. 2, b_i = int f phi_i) -------------------------------
 * fq: device float64 [ne][q1d^3] ([ne][q1d^2] in 2D), source values at the form's quadrature
 * points; b: device float64 [ndof], overwritten with
 * b_i = sum_e sum_q w_q det J_q fq(e,q) phi_i(q). */
fem_status fem_rhs(const fem_form* form, const double* fq, double* b, void* stream);
/* Physical coordinates of the quadrature points: xq device float64
 * [ne][q1d^3][3] ([ne][q1d^2][2] in 2D). */
fem_status fem_qpoint_coords(const fem_form* form, double* xq, void* stream);

/* ---- Jacobi-preconditioned CG (Sec. 5.2, CGSolver with SetRelTol /
 * SetMaxIter) -----------------------------------------------------------------
 * Solves A_c x = b for the constrained operator. On entry x holds the initial
 * guess including the essential values g on essential DOFs; b must already be
 * the constrained right-hand side (b_ess = g, b_free = b - A g on free DOFs;
 * fem_lift_rhs builds it). Stops when ||b - A_c x||_2 <= rtol ||b||_2 for the
 * true residual (recomputed in FP64 at exit; the iteration restarts from x if
 * the recursive residual drifted). precision FEM_SOLVE_MIXED runs FP32 inner
 * Jacobi-PCG to inner_rtol on FP32 copies of D, inside FP64 iterative
 * refinement (FP64 outer residual, norms and updates; a pass that needs less
 * than inner_rtol to reach the tolerance stops at half of it).
 * precond FEM_PC_NONE replaces the Jacobi diagonal by ones.
 * Synchronises `stream`. Errors: FEM_ENOCONV, FEM_EBREAKDOWN. */
typedef struct {
  double rtol;          /* relative tolerance, e.g. 1e-10 */
  int maxit;            /* cap on (inner, for mixed) CG iterations */
  int precision;        /* FEM_SOLVE_F64 or FEM_SOLVE_MIXED */
  double inner_rtol;    /* mixed: inner relative tolerance; reliable updates:
                           residual drop between updates; <= 0 (the default)
                           takes the measured default of the call and mode:
                           fem_solve 1e-4 (FEM_SOLVE_MIXED), 0.1
                           (FEM_SOLVE_MIXED_RU); fem_mg_solve 3e-4;
                           fem_batch_solve 1e-4 */
  int max_outer;        /* mixed: cap on refinement steps */
  int check_every;      /* iterations per CUDA-graph launch between host polls */
  int use_graph;        /* capture check_every iterations in a CUDA graph */
  int precond;          /* FEM_PC_JACOBI (default) or FEM_PC_NONE (plain CG) */
} fem_solve_opts;
typedef struct {
  int iterations;       /* total CG iterations (inner iterations for mixed) */
  int outer;            /* refinement steps (mixed) or restarts (FP64) */
  int converged;        /* 1 if the true residual met rtol */
  double relres;        /* final ||b - A_c x||_2 / ||b||_2, FP64 */
  double bnorm;         /* ||b||_2 */
} fem_solve_info;
void fem_solve_opts_default(fem_solve_opts* opts);
fem_status fem_solve(const fem_form* form, const double* b, double* x,
                     const fem_solve_opts* opts, fem_solve_info* info, void* stream);
/* b_c = (I-E)(b - A g) + E g for the essential values held in g on essential
 * DOFs (g is read on essential DOFs only). b, g, bc: device float64 [ndof]. */
fem_status fem_lift_rhs(const fem_form* form, const double* b, const double* g,
                        double* bc, void* stream);

/* ---- compliance gradient (differentiation; the paper's LiDO application,
 * Sec. 7, motivates it; no kernel in the paper) ------------------------------
 * For a diffusion form: g_e = -(1/coef_e) sum_q gradhat(u)^T D_q gradhat(u)
 * = -u_e^T Khat_e u_e, the derivative of J = b^T u (A u = b, b independent of
 * the coefficient, self-adjoint so the adjoint state is u) with respect to
 * coef_e. u: device float64 [ndof] (zero on essential DOFs); g: device
 * float64 [ne]. */
fem_status fem_compliance_grad(const fem_form* form, const double* u, double* g,
                               void* stream);
/* Compliance J = b^T u (deterministic fixed-order FP64 reduction) into J, a
 * device float64 scalar. b, u: device float64 [ndof]. */
fem_status fem_compliance(const fem_form* form, const double* b, const double* u, double* J,
                          void* stream);

/* ---- batching: many independent problems, several right-hand sides each --
 * (no batched path in the paper; it extends the element-parallel apply of
 * Sec. 4.3 across problems). A batch refers to nprob forms (any mix of orders,
 * sizes and kinds; they must outlive the batch) and nrhs right-hand sides per
 * problem. Batched vectors are concatenated problem after problem; problem
 * i's block is [nrhs][ndof_i] and starts at nrhs * off[i], off[i] = sum of
 * ndof_j for j < i (fem_batch_info). System s = i * nrhs + r.
 * The element phase is one persistent kernel over (problem, element tile)
 * work items, each applying its tile to all nrhs right-hand sides (D streams
 * from HBM once per nrhs); the scatter is one persistent kernel over
 * (problem, DOF chunk) items. Applies and CG iterations run as CUDA graphs.
 * Problems on hexahedral and quadrilateral meshes may be mixed (a 2D tile
 * puts one element on each row of q1d threads). Orders p = 1..6
 * (FEM_EUNSUPPORTED otherwise). */
fem_status fem_batch_create(const fem_form* const* forms, int nprob, int nrhs, void* stream,
                            fem_batch** out);
void fem_batch_destroy(fem_batch* batch);
/* total_len = nrhs * sum ndof; off_host [nprob + 1] (may be NULL). */
fem_status fem_batch_info(const fem_batch* batch, int64_t* total_len, int64_t* off_host);
/* Y = A X (or A_c X when constrained != 0: every form needs its essential
 * DOFs) for all systems; dtype FEM_F64 or FEM_F32 (float copies of D are made
 * on first use). X, Y: device arrays of total_len entries, not aliased. The
 * launches are captured once per (X, Y, dtype, constrained) into a CUDA
 * graph that later calls replay. */
fem_status fem_batch_apply(fem_batch* batch, int dtype, const void* X, void* Y, int constrained,
                           void* stream);
/* Jacobi-PCG for every system (all systems advance together; converged ones
 * idle), with the stopping rule and precision options of fem_solve applied
 * per system. B: constrained right-hand sides; X: initial guesses including
 * essential values (overwritten). iters_host [nsys] and relres_host [nsys]
 * receive per-system iterations and final true relative residuals (either
 * may be NULL). Synchronises stream. Errors: FEM_ENOCONV, FEM_EBREAKDOWN. */
fem_status fem_batch_solve(fem_batch* batch, const double* B, double* X, const fem_solve_opts* opts,
                           int* iters_host, double* relres_host, void* stream);
/* Autotuner: for every (p, q) of the batch's hexahedral problems, times the
 * batched apply with candidate element tiles (elements per work item) and
 * keeps the fastest (quadrilateral problems keep floor(256 / q1d));
 * results are read from / written to the line-per-entry JSON cache at
 * cache_path (NULL: no cache), keyed by device name, dtype and (p, q). */
fem_status fem_batch_tune(fem_batch* batch, int dtype, const char* cache_path, void* stream);
/* Current element tiles of the hexahedral problems: tiles_host [18], entry
 * 2p + (q - p - 1). */
fem_status fem_batch_tiles(const fem_batch* batch, int* tiles_host);

/* ---- p-multigrid preconditioner (Sec. 5.2 names matrix-free p-multigrid
 * for PA operators as a research direction without fixing an algorithm; the
 * algorithm below is this library's) --------------------------------------
 * Levels p, p/2, ..., 1 on the fine form's mesh and coefficient, each a PA
 * form of the same kind with q_l = p_l + (q - p) points. A coarse DOF is
 * essential iff every fine DOF of the same mesh entity is. Transfers: P =
 * nodal interpolation of the coarse function at the fine GLL nodes (each
 * fine DOF takes its value from the first element holding it), masked to
 * free DOFs on both sides; restriction = P^T. Smoother: cheb_order steps of
 * Jacobi-preconditioned Chebyshev iteration on [cheb_lo, 1] * cheb_hi *
 * lambda, lambda = D-Rayleigh quotient after power_its power iterations on
 * D^-1 A_c from v_i = frac(i * 2654435761 / 2^32) - 1/2 (A_c applied in
 * double-float, FP64 vectors and dot products). Coarsest level:
 * coarse_its Jacobi-PCG iterations from zero. V-cycle: pre-smoothing from
 * zero, restricted residual, recursion, prolongated correction,
 * post-smoothing. 3D (hexahedral) forms only. Elasticity forms: every
 * level is an elasticity form with the same Lame coefficients, the
 * essential rule and the transfers act on each component (P is
 * block-diagonal over the components of component-major vectors), and
 * all vectors below are [3 ndof] of their level. Convection forms are
 * rejected (FEM_EINVAL). */
typedef struct fem_mg fem_mg;
typedef struct {
  int cheb_order;       /* Chebyshev steps per pre- and post-smoothing (2) */
  double cheb_lo;       /* lower end of the smoothing interval / upper end (0.25) */
  double cheb_hi;       /* upper end / estimated lambda_max of D^-1 A_c (1.1) */
  int power_its;        /* power iterations per smoothed level (20) */
  int coarse_its;       /* Jacobi-PCG iterations on the coarsest level (30) */
  int precision;        /* FEM_F64 or FEM_F32: arithmetic of the V-cycle */
  int coarse_assembled; /* 1: an order-1 coarsest level of a scalar form is
                           assembled once into a sparse matrix (CSR, entries
                           summed in ascending element order) that its CG
                           multiplies by; 0: matrix-free like every other
                           level (1) */
} fem_mg_opts;
void fem_mg_opts_default(fem_mg_opts* opts);
/* Builds the hierarchy for `fine` (fem_form_set_essential must have been
 * called on it; the handle keeps a pointer to it: keep it alive and do not
 * change its coefficient or essential DOFs while the handle exists). The
 * coarse spaces and forms, diagonals, FP32 copies (precision FEM_F32) and
 * lambda estimates are made here, synchronously on `stream`. Errors:
 * FEM_EINVAL (bad options, no essential list), FEM_EUNSUPPORTED (2D mesh),
 * FEM_ENOMEM. */
fem_status fem_mg_create(const fem_form* fine, const fem_mg_opts* opts, void* stream,
                         fem_mg** out);
void fem_mg_destroy(fem_mg* mg);
/* Level count and, per level l (fine first), order, lambda estimate (0 on
 * the coarsest level) and vector length (DOF count times the form's
 * components); each host array may be NULL or holds
 * at least nlevels entries. */
fem_status fem_mg_info(const fem_mg* mg, int* nlevels, int* orders_host,
                       double* lambdas_host, int64_t* ndofs_host);
/* One V-cycle: z = M^-1 r. r, z: device float64 [ndof] of the fine space;
 * entries of r on essential DOFs are ignored (taken as 0), z is 0 there.
 * Uses the fine form's E-vector scratch: do not run another operation of
 * that form concurrently. */
fem_status fem_mg_vcycle(fem_mg* mg, const double* r, double* z, void* stream);
/* The form of level l (0 = the fine form); owned by the handle (level 0 by
 * the caller). Its essential DOFs are the level's. NULL if l is out of
 * range. */
const fem_form* fem_mg_level_form(const fem_mg* mg, int level);
/* Transfers between level l (finer) and l + 1, FP64: zf = P~ zc (prolong)
 * and rc = P~^T rf (restrict), with P~ = (I - E_l) P (I - E_{l+1}). zc, rc:
 * device float64 [ndof of level l+1]; zf, rf: [ndof of level l]. Uses the
 * E-vector scratch of both levels' forms. Errors: FEM_EINVAL (l out of
 * range). */
fem_status fem_mg_prolong(fem_mg* mg, int level, const double* zc, double* zf, void* stream);
fem_status fem_mg_restrict(fem_mg* mg, int level, const double* rf, double* rc, void* stream);
/* Flexible CG (FP64; beta = z.(r - r_old) / z_old.r_old) on the fine
 * constrained operator, preconditioned by one V-cycle per iteration. x and b
 * as for fem_solve; opts: rtol, maxit, max_outer (restarts when the true
 * residual disagrees with the recursive one), check_every, use_graph, and
 * precision, the arithmetic of the outer operator apply: FEM_SOLVE_F64,
 * FEM_SOLVE_DF64, or FEM_SOLVE_MIXED (the FP32 operator, p and q rounded to
 * FP32 around it, inside FP64 iterative refinement: each pass runs until the
 * recursive residual has dropped by inner_rtol, then restarts from the FP64
 * true residual); the final true residual is always FP64; the other fields
 * are ignored. The essential entries of the initial guess are replaced by
 * those of b (A_c x = b fixes them; the V-cycle never corrects them).
 * Synchronises `stream`. Errors: FEM_EINVAL (other precision), FEM_ENOCONV,
 * FEM_EBREAKDOWN. */
fem_status fem_mg_solve(fem_mg* mg, const double* b, double* x, const fem_solve_opts* opts,
                        fem_solve_info* info, void* stream);

/* ---- sharded operator: element partition with an owned + halo L-vector --
 * The paper's parallel operator is A = P^T G^T B^T D B G P (Sec. 4.3
 * "Operator Decomposition"): every rank applies G^T B^T D B G to the
 * elements it owns, and P / P^T move values between the global true-DOF
 * vector and the ranks' local L-vectors -- the parallel assembly step that
 * FormLinearSystem performs (Sec. 5.1). Here a rank's L-vector holds every
 * DOF of its elements (owned ones and a halo of DOFs shared with other
 * ranks), and vectors are kept consistent: each shared DOF has the same value
 * on every rank that holds it. After a rank's element kernel and scatter,
 * each shared DOF holds this rank's partial sum only; one exchange with the
 * neighbouring ranks (each sends its partials of the DOFs it shares with that
 * neighbour) and a combine step that adds the partials of all sharing ranks
 * in ascending rank order give every holder the same assembled value (P^T
 * then P in one round). Dot products count each DOF once, on its owner (the
 * lowest rank holding it), and sum the ranks' results with an all-reduce.
 *
 * Communication belongs to the caller (NCCL, gloo, MPI ...), through the
 * callbacks of fem_comm. Exchange buffers are device float64 arrays owned by
 * the shard, laid out neighbour after neighbour; for neighbour k the
 * vdim * count_k values run from off[k] to off[k+1], component-major inside
 * that range, DOFs in ascending global number (the same order on both ends).
 * The library synchronises `stream` before a callback when host_sync != 0
 * (transports that read device memory from the host); otherwise the callback
 * must order its work after the work already on `stream` and before work
 * enqueued later (as torch.distributed's NCCL backend does on the current
 * stream). A callback returns 0 on success; anything else makes the calling
 * entry point fail with FEM_ECUDA. */
typedef struct fem_comm {
  void* ctx;
  int host_sync;
  /* Send send[off[k], off[k+1]) to rank nbr[k] and receive the same number
   * of values from it into recv[off[k], off[k+1]), for k < nnbr. nbr and off
   * are host arrays owned by the shard; send and recv are device pointers. */
  int (*exchange)(void* ctx, int nnbr, const int32_t* nbr, const int64_t* off, double* send, double* recv,
                  void* stream);
  /* Sum vals[0, n) (device float64) over all ranks, in place. */
  int (*allreduce)(void* ctx, double* vals, int n, void* stream);
} fem_comm;

typedef struct fem_shard fem_shard;

/* Element partition into nparts slabs: elements sorted by the centroid of
 * their vertices along the coordinate axis in which the centroids spread
 * widest (ties by element number), then cut into nparts runs of consecutive
 * elements, the first ne % nparts runs one element longer. part_host[ne]
 * (host, caller-owned) receives each element's part. The same mesh gives
 * the same partition on every rank. Errors: FEM_EINVAL (nparts < 1 or
 * nparts > ne). */
fem_status fem_partition_slabs(const fem_mesh* mesh, int nparts, int32_t* part_host);

/* Rank `rank`'s shard of the global space gspace under the element
 * partition part_host[ne] (values in [0, nparts), nparts <= 64): its
 * elements in ascending global number, a local mesh of their vertices
 * (ascending global vertex number), the local space of order p on it (its
 * own numbering, Sec. 3.4), the local -> global DOF map, ownership, the
 * neighbour ranks, and the exchange and combine tables (uploaded to the
 * device). Forms for the shard are created on fem_shard_space(). Every rank
 * builds the same global space to agree on global DOF numbers. Errors:
 * FEM_EINVAL (arguments, a rank without elements), FEM_EUNSUPPORTED
 * (curved meshes), FEM_ENOMEM. */
fem_status fem_shard_create(const fem_space* gspace, const int32_t* part_host, int nparts, int rank,
                            fem_shard** out);
void fem_shard_destroy(fem_shard* sh);
/* The shard's local space (owned by the shard; valid until it is
 * destroyed). */
const fem_space* fem_shard_space(const fem_shard* sh);
/* Sizes: local elements, local DOFs, owned local DOFs, neighbour ranks,
 * exchange slots (DOFs shared with a neighbour, summed over neighbours),
 * and global DOFs; any pointer may be NULL. */
fem_status fem_shard_info(const fem_shard* sh, int64_t* ne_local, int64_t* ndof_local, int64_t* ndof_owned,
                          int* nnbr, int64_t* nslots, int64_t* ndof_global);
/* Host copies of the plan (any pointer may be NULL): elems[ne_local] global
 * element numbers; l2g[ndof_local] global DOF of each local DOF;
 * owned[ndof_local] 1 where this rank owns the DOF; nbr[nnbr] neighbour
 * ranks, ascending; slot_off[nnbr + 1] slot ranges per neighbour;
 * slot_dof[nslots] local DOF of each slot (per neighbour in ascending
 * global DOF order). */
fem_status fem_shard_tables(const fem_shard* sh, int64_t* elems, int64_t* l2g, uint8_t* owned, int32_t* nbr,
                            int64_t* slot_off, int32_t* slot_dof);
/* Combine table (host copies): for the nshared local DOFs held by more than
 * one rank, comb_dof[j] is the local DOF and comb_off[j] .. comb_off[j+1]
 * its entries in ascending rank order, comb_src[t] = -1 for this rank's own
 * partial, else the slot holding the partial received from that rank. Any
 * pointer may be NULL; *nshared and *nentries give the sizes. */
fem_status fem_shard_combine_table(const fem_shard* sh, int64_t* nshared, int64_t* nentries, int32_t* comb_dof,
                                   int32_t* comb_off, int32_t* comb_src);
/* Map global DOF numbers (host, n) to local ones: out_host[i] = local DOF of
 * global_host[i], or -1 when this shard does not hold it. */
fem_status fem_shard_localize(const fem_shard* sh, const int32_t* global_host, int64_t n, int32_t* out_host);
/* Device gathers between a global vector (length vdim * ndof_global,
 * component-major) and the local one (vdim * ndof_local): to_local copies
 * every local entry from its global DOF; to_global writes the owned local
 * entries into the global vector (other entries untouched). */
fem_status fem_shard_to_local(const fem_shard* sh, int vdim, const double* xg, double* xl, void* stream);
fem_status fem_shard_to_global(const fem_shard* sh, int vdim, const double* xl, double* xg, void* stream);
/* y = A x on consistent local L-vectors (float64, vdim * ndof_local) with
 * the form `form` created on fem_shard_space(sh): element kernel and scatter
 * of the local elements, exchange of the shared DOFs' partials, combine;
 * constrained != 0 applies A_c as fem_apply does (needs the form's essential
 * DOFs: the local numbers of the global essential set, fem_shard_localize).
 * Errors: as fem_apply, FEM_ECUDA when a callback fails. */
fem_status fem_shard_apply(const fem_shard* sh, const fem_form* form, const double* x, double* y, int constrained,
                           const fem_comm* comm, void* stream);
/* Assembled diagonal (consistent), constrained as fem_assemble_diagonal. */
fem_status fem_shard_diagonal(const fem_shard* sh, const fem_form* form, double* diag, int constrained,
                              const fem_comm* comm, void* stream);
/* Load vector b from quadrature-point values of the local elements
 * (fq [ne_local][q1d^3], as fem_rhs), assembled across ranks. */
fem_status fem_shard_rhs(const fem_shard* sh, const fem_form* form, const double* fq, double* b,
                         const fem_comm* comm, void* stream);
/* *out_host = sum over owned entries of a . b, summed over ranks (all
 * vectors consistent, vdim * ndof_local). Synchronises `stream`. */
fem_status fem_shard_dot(const fem_shard* sh, int vdim, const double* a, const double* b, double* out_host,
                         const fem_comm* comm, void* stream);
/* Jacobi-PCG (FP64) on the sharded constrained operator, the iteration of
 * fem_solve: x0 = x (its essential entries are the Dirichlet values), stop
 * when the true residual ||b - A_c x|| <= rtol ||b|| (confirmed at exit).
 * Per iteration: one sharded apply (one exchange) and two all-reduces (p.q;
 * then r.z and r.r together). opts: rtol, maxit, max_outer (restarts from
 * the true residual), precond; other fields are ignored (FP64 only).
 * Synchronises `stream`; fills info. Errors: as fem_solve. */
fem_status fem_shard_solve(const fem_shard* sh, const fem_form* form, const double* b, double* x,
                           const fem_solve_opts* opts, fem_solve_info* info, const fem_comm* comm, void* stream);

/* ---- arithmetic-peak probe (the paper has no counterpart) ---------------
 * Measures the fused multiply-add rate of the current device in the given
 * arithmetic: one kernel on every SM at full occupancy, eight independent
 * FMA chains per thread, `iters` steps per chain, timed with CUDA events on
 * `stream` (best of three after one warm-up launch). *tflops receives
 * 2 * chains * iters * threads / seconds / 1e12 (an FMA counts two flops).
 * These are the denominators of the roofline fractions of the kernels bound
 * by their arithmetic pipe (the FP64 element kernels; double-float and FP32
 * run on the FP32 pipe). dtype: FEM_F64 or FEM_F32. Synchronises `stream`.
 * A run of about 20 ms: iters ~ 5,000 (FP64), ~ 300,000 (FP32) on GB300.
 * Errors: FEM_EINVAL (dtype, iters <= 0, NULL tflops), FEM_ECUDA. */
fem_status fem_probe_fma_peak(int dtype, int iters, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FEM_H */
