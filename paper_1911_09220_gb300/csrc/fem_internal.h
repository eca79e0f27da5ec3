// Internal declarations shared by the library's host and CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "fem.h"

// ---------------------------------------------------------------- errors ----
fem_status fem_fail(fem_status st, const char* fmt, ...);
#define FEM_TRY(expr)                          \
  do {                                         \
    fem_status _st = (expr);                   \
    if (_st != FEM_OK) return _st;             \
  } while (0)
#define FEM_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess)                                                          \
      return fem_fail(FEM_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,         \
                      cudaGetErrorString(_e));                                      \
  } while (0)
#define FEM_LAUNCHED() FEM_CUDA(cudaGetLastError())

// Device buffer helpers (library-owned memory).
template <typename T>
fem_status dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return FEM_OK;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fem_fail(FEM_ENOMEM, "cudaMalloc(%zu bytes): %s", count * sizeof(T),
                    cudaGetErrorString(e));
  }
  return FEM_OK;
}
template <typename T>
void dev_free(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// ---------------------------------------------------------------- handles ---
struct fem_mesh {
  int dim = 3;                  // 3: hexahedra, 2: quadrilaterals
  int nvpe = 8;                 // vertices per element (8 or 4)
  int64_t nv = 0, ne = 0;
  std::vector<double> coords;   // [nv][dim]
  std::vector<int32_t> hex;     // [ne][nvpe] element vertex tuples
  double* d_coords = nullptr;
  int32_t* d_hex = nullptr;
  // optional order-k nodal geometry (Sec. 3.1 "nodes"): [ne][(k+1)^3][3]
  int geo_k = 0;
  double* d_gnodes = nullptr;
  // hexahedral topology shared by every space on the mesh (built by the
  // first fem_space_create): edge and face ids in order of first appearance
  // per (element, local edge / face) slot
  mutable std::mutex topo_mu;
  mutable bool topo_done = false;
  mutable int64_t n_edges = 0, n_faces = 0;
  mutable std::vector<int32_t> edge_id, face_id;  // [ne][12], [ne][6]
};

struct fem_space {
  const fem_mesh* mesh = nullptr;
  int p = 0, D1 = 0, nd = 0;    // nd = D1^3 local DOFs
  int64_t ne = 0, ndof = 0;
  int64_t n_edges = 0, n_faces = 0;
  std::vector<int32_t> e2l;     // [ne][nd]
  std::vector<int32_t> bdr;     // boundary DOFs, ascending
  std::vector<double> nodes;    // GLL nodes on [0,1], D1
  int32_t* d_e2l = nullptr;     // [ne][nd]
  int32_t* d_l2e_off = nullptr; // [ndof+1]
  int32_t* d_l2e_idx = nullptr; // [ne*nd], e*nd + k
  int32_t* d_pos = nullptr;     // [ne*nd]: position of slot e*nd + k in the inverse map (DOF-sorted order)
  double* d_nodes = nullptr;
  double* d_gBn = nullptr;      // order-k geometry basis at this space's GLL nodes [D1][k+1]
  int gBn_k = 0;
};

struct fem_form {
  const fem_space* space = nullptr;
  int kind = FEM_DIFFUSION;
  int q1d = 0, nq = 0, ncomp = 0;  // nq = q1d^3; ncomp 6, 3, 1 or 12 (elasticity)
  int vdim = 1;                    // vector components per DOF (3 for elasticity)
  double* d_coef = nullptr;        // [ne] (elasticity: lambda)
  double* d_mu = nullptr;          // elasticity: mu [ne]
  double* d_D = nullptr;           // [ne][ncomp][nq]
  float* d_D32 = nullptr;          // lazily made float copy
  double* d_B = nullptr;           // [q1d][D1] basis values at Gauss points
  double* d_G = nullptr;           // [q1d][D1] derivatives
  float* d_B32 = nullptr;
  float* d_G32 = nullptr;
  float* d_Bdf = nullptr;          // [q1d][D1] double-float pairs (hi, lo)
  float* d_Gdf = nullptr;
  float* d_Ddf = nullptr;          // lazily made double-float copy of D (pairs)
  double* d_qpts = nullptr;        // [q1d]
  double* d_qwts = nullptr;        // [q1d]
  void* d_ye = nullptr;            // E-vector scratch, ne*nd doubles
  uint8_t* d_ess_mask = nullptr;   // [ndof], 1 on essential DOFs
  int32_t* d_ess = nullptr;
  int64_t n_ess = 0;
  int* d_flag = nullptr;           // device status word for setup checks
  // solver workspace (lazy)
  double* d_work64 = nullptr;
  size_t work64_len = 0;
  float* d_work32 = nullptr;
  size_t work32_len = 0;
  double* d_red = nullptr;         // reduction partials / scalars
  size_t red_len = 0;
  int* h_pinned = nullptr;         // pinned host status words
  double* d_beta = nullptr;        // convection: velocity [ne][nq][3]
  // order-k geometry basis at this form's Gauss points, [q1d][k+1] (curved meshes)
  double* d_gB = nullptr;
  double* d_gG = nullptr;
  int geo_k = 0;
};

// Rank `rank`'s part of an element-partitioned space (fem_shard.cpp builds
// the plan on the host; k_shard.cu runs the exchange-side kernels and the
// sharded solver).
struct fem_shard {
  int nparts = 1, rank = 0;
  int64_t ndof_global = 0;
  fem_mesh* lmesh = nullptr;            // owned local mesh and space
  fem_space* lspace = nullptr;
  std::vector<int64_t> elems;           // global element numbers, ascending
  std::vector<int64_t> l2g;             // [ndof_local] global DOF
  std::vector<uint8_t> owned;           // [ndof_local]
  int64_t n_owned = 0;
  std::vector<int32_t> nbr;             // neighbour ranks, ascending
  std::vector<int64_t> slot_off;        // [nnbr + 1] slot ranges per neighbour
  std::vector<int32_t> slot_dof;        // [nslots] local DOF per slot
  std::vector<int32_t> comb_dof, comb_off, comb_src;  // combine table (see fem.h)
  // exchange buffer offsets for vdim = 1 and 3: [nnbr + 1] in doubles
  std::vector<int64_t> xoff1, xoff3;
  // device copies
  int64_t* d_l2g = nullptr;
  uint8_t* d_owned = nullptr;
  int32_t* d_slot_dof = nullptr;
  int32_t* d_slot_nbr = nullptr;        // [nslots] neighbour index of each slot
  int64_t* d_slot_off = nullptr;        // [nnbr + 1]
  int32_t* d_comb_dof = nullptr;
  int32_t* d_comb_off = nullptr;
  int32_t* d_comb_src = nullptr;
  double* d_send = nullptr;             // 3 * nslots (room for vector forms)
  double* d_recv = nullptr;
  // solver workspace (lazy, k_shard.cu)
  mutable double* d_work = nullptr;
  mutable size_t work_len = 0;
  mutable double* d_red = nullptr;
  mutable size_t red_len = 0;
  mutable double* h_pinned = nullptr;
};

// Length of the form's vectors: vdim * ndof (component-major).// Length of the form's vectors: vdim * ndof (component-major).
inline int64_t fem_form_len(const fem_form* f) { return (int64_t)f->vdim * f->space->ndof; }
// opts.inner_rtol, or, when it is <= 0, the default of fem_solve (which 0;
// by precision), fem_mg_solve (1) or fem_batch_solve (2); k_solve.cu.
double fem_inner_rtol(const fem_solve_opts& o, int which);

// ---------------------------------------------------------------- basis -----
// 1D tables on [0,1]: GLL nodes (D1 = p+1), Gauss-Legendre points/weights (q),
// B[k][j] = l_j(x_k), G[k][j] = l_j'(x_k) for GLL Lagrange polynomials l_j.
void fem_gll_nodes(int p, std::vector<double>& nodes);
void fem_gauss_rule(int q, std::vector<double>& pts, std::vector<double>& wts);
void fem_lagrange_tables(const std::vector<double>& nodes, const std::vector<double>& pts,
                         std::vector<double>& B, std::vector<double>& G);

// ---------------------------------------------------------------- kernels ---
int fem_kernels_supported(int p, int q1d);
fem_status fem_launch_setup(const fem_form* f, cudaStream_t s);
fem_status fem_launch_qpoint_coords(const fem_form* f, double* xq, cudaStream_t s);
fem_status fem_launch_dof_coords(const fem_space* sp, double* out, cudaStream_t s);
// sorted: the element kernel writes each E-vector value at its slot's
// position in the inverse map (DOF-sorted order, space->d_pos) instead of
// e*nd + k, and the scatter then reads each DOF's values contiguously. The
// two halves must agree; fem_sorted_evec(f, dtype) says whether a form uses
// it (3D forms whose E-vector exceeds half the L2; a vector form sorts each
// component's block), and both launchers fall back to the element-major
// order otherwise. dtype: the element dtype (FEM_DF64 E-vectors are float64).
fem_status fem_launch_apply_element(const fem_form* f, int dtype, const void* x, void* ye,
                                    cudaStream_t s, const int* skip = nullptr, bool sorted = false);
// scatter: y_i = sum over inverse map of ye; ess rows (if mask) get x_i (constrained).
// pdot != nullptr: also writes per-block partial sums of x_i*y_i to pdot[nblocks].
fem_status fem_launch_scatter(const fem_form* f, int dtype, const void* ye, void* y,
                              const uint8_t* mask, const void* xess, double* pdot,
                              int nblocks, cudaStream_t s, const int* skip = nullptr, bool sorted = false);
bool fem_sorted_evec(const fem_form* f, int dtype);
fem_status fem_launch_zero_ess(const fem_form* f, int dtype, const void* x, void* xz,
                               cudaStream_t s);
fem_status fem_launch_diag_element(const fem_form* f, double* ye, cudaStream_t s);
// Elasticity element kernel (k_elasticity.cu) and its diagonal helper: the
// 6-component matrix of component c at every point, [ne][q1d^3][6].
fem_status fem_launch_apply_elasticity(const fem_form* f, int dtype, const void* x, void* ye, cudaStream_t s,
                                       const int* skip, bool sorted = false);
fem_status fem_launch_elasticity_diag_D(const fem_form* f, int c, double* Dc, cudaStream_t s);
fem_status fem_launch_rhs_element(const fem_form* f, const double* fq, double* ye,
                                  cudaStream_t s);
fem_status fem_launch_grad(const fem_form* f, const double* u, double* g, cudaStream_t s);
fem_status fem_form_ensure_f32(const fem_form* f, cudaStream_t s);
fem_status fem_form_ensure_df64(const fem_form* f, cudaStream_t s);
fem_status fem_launch_mark_ess(const fem_form* f, cudaStream_t s);
int fem_scatter_blocks(int64_t ndof);
// Constant-memory 1D tables of the element kernels (one copy per translation
// unit): filled once per device from form / batch creation.
fem_status fem_apply_tables_init();
fem_status fem_batch_tables_init();
fem_status fem_2d_tables_init();
fem_status fem_elast_tables_init();
// Quadrilateral (2D) counterparts, dispatched on mesh->dim == 2 (k_2d.cu).
fem_status fem_launch_setup_2d(const fem_form* f, cudaStream_t s);
fem_status fem_launch_qpoint_coords_2d(const fem_form* f, double* xq, cudaStream_t s);
fem_status fem_launch_dof_coords_2d(const fem_space* sp, double* out, cudaStream_t s);
fem_status fem_launch_apply_element_2d(const fem_form* f, int dtype, const void* x, void* ye, cudaStream_t s,
                                       const int* skip);
fem_status fem_launch_diag_element_2d(const fem_form* f, double* ye, cudaStream_t s);
fem_status fem_launch_rhs_element_2d(const fem_form* f, const double* fq, double* ye, cudaStream_t s);
fem_status fem_launch_grad_2d(const fem_form* f, const double* u, double* g, cudaStream_t s);
// p-multigrid coarse essential DOFs (host; fem_host.cpp): a coarse DOF is
// essential iff every fine DOF of the same mesh entity is. essf: fine mask of
// one component [sf->ndof]; returns coarse ids, ascending.
std::vector<int32_t> fem_coarse_essential(const fem_space* sf, const uint8_t* essf, const fem_space* sc);
// Make the form's geometry tables match its mesh's nodal order (no-op for
// vertex-only meshes); synchronous.
fem_status fem_form_geo_tables(const fem_form* f);
