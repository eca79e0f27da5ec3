// Partial-assembly setup: quadrature data D at every element and Gauss point
// (Sec. 4.3, "setup phase that evaluates and stores D"), plus coordinate
// helpers (quadrature points, DOF nodes) and the essential-DOF mask.
#include "fem_internal.h"
#include "k_common.cuh"

namespace {

// Trilinear map of one hexahedron (Sec. 3.1, Eq. mesh_eq_x with the 8 vertex
// coordinates and trilinear w_i on [0,1]^3).
struct Hex8 {
  double X[8][3];
  __device__ void load(const double* __restrict__ coords, const int32_t* __restrict__ hex, int64_t e) {
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int32_t g = hex[8 * e + v];
#pragma unroll
      for (int d = 0; d < 3; ++d) X[v][d] = coords[3 * (int64_t)g + d];
    }
  }
  // corner v has reference coordinates (cx, cy, cz) with cx = (v==1||v==2||v==5||v==6) etc.
  __device__ static int cx(int v) { return (v == 1 || v == 2 || v == 5 || v == 6); }
  __device__ static int cy(int v) { return (v == 2 || v == 3 || v == 6 || v == 7); }
  __device__ static int cz(int v) { return v >= 4; }
  __device__ void map(double a, double b, double c, double x[3]) const {
    x[0] = x[1] = x[2] = 0.0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const double N = (cx(v) ? a : 1.0 - a) * (cy(v) ? b : 1.0 - b) * (cz(v) ? c : 1.0 - c);
#pragma unroll
      for (int d = 0; d < 3; ++d) x[d] += N * X[v][d];
    }
  }
  // J[r][c] = d x_r / d xhat_c
  __device__ void jacobian(double a, double b, double c, double J[3][3]) const {
#pragma unroll
    for (int r = 0; r < 3; ++r) J[r][0] = J[r][1] = J[r][2] = 0.0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const double fa = cx(v) ? a : 1.0 - a, da = cx(v) ? 1.0 : -1.0;
      const double fb = cy(v) ? b : 1.0 - b, db = cy(v) ? 1.0 : -1.0;
      const double fc = cz(v) ? c : 1.0 - c, dc = cz(v) ? 1.0 : -1.0;
      const double g0 = da * fb * fc, g1 = fa * db * fc, g2 = fa * fb * dc;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        J[r][0] += X[v][r] * g0;
        J[r][1] += X[v][r] * g1;
        J[r][2] += X[v][r] * g2;
      }
    }
  }
};

// One thread per (element, quadrature point).
//   diffusion: D = coef * w * adj(J) adj(J)^T / det J  (= coef w det J J^-1 J^-T),
//              components 00,01,02,11,12,22;
//   mass:      D = coef * w * det J.
__global__ void k_setup(int64_t ne, int Q, int kind, const double* __restrict__ coords,
                        const int32_t* __restrict__ hex, const double* __restrict__ qpts,
                        const double* __restrict__ qwts, const double* __restrict__ coef,
                        double* __restrict__ Dout, int* __restrict__ flag) {
  const int nq = Q * Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq);
    const int q1 = q % Q, q2 = (q / Q) % Q, q3 = q / (Q * Q);
    Hex8 h;
    h.load(coords, hex, e);
    double J[3][3];
    h.jacobian(qpts[q1], qpts[q2], qpts[q3], J);
    // cofactors C[r][c]; adj(J)[a][b] = C[b][a]
    double C[3][3];
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]);
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = -(J[0][1] * J[2][2] - J[0][2] * J[2][1]);
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = -(J[0][0] * J[2][1] - J[0][1] * J[2][0]);
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = -(J[0][0] * J[1][2] - J[0][2] * J[1][0]);
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    if (!(det > 0.0)) {
      if (atomicExch(&flag[0], 1) == 0) flag[1] = (int)e;
    }
    const double w = qwts[q1] * qwts[q2] * qwts[q3] * coef[e];
    if (kind == FEM_DIFFUSION) {
      const double s = w / det;
      // D_ab = s * sum_c adj[a][c] adj[b][c] = s * sum_c C[c][a] C[c][b]
      // point-major: the six components of a point are contiguous
      double* De = Dout + (e * nq + q) * 6;
      De[0] = s * (C[0][0] * C[0][0] + C[1][0] * C[1][0] + C[2][0] * C[2][0]);
      De[1] = s * (C[0][0] * C[0][1] + C[1][0] * C[1][1] + C[2][0] * C[2][1]);
      De[2] = s * (C[0][0] * C[0][2] + C[1][0] * C[1][2] + C[2][0] * C[2][2]);
      De[3] = s * (C[0][1] * C[0][1] + C[1][1] * C[1][1] + C[2][1] * C[2][1]);
      De[4] = s * (C[0][1] * C[0][2] + C[1][1] * C[1][2] + C[2][1] * C[2][2]);
      De[5] = s * (C[0][2] * C[0][2] + C[1][2] * C[1][2] + C[2][2] * C[2][2]);
    } else {
      Dout[e * nq + q] = w * det;
    }
  }
}

__global__ void k_qpoint_coords(int64_t ne, int Q, const double* __restrict__ coords,
                                const int32_t* __restrict__ hex, const double* __restrict__ qpts,
                                double* __restrict__ xq) {
  const int nq = Q * Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq);
    Hex8 h;
    h.load(coords, hex, e);
    double x[3];
    h.map(qpts[q % Q], qpts[(q / Q) % Q], qpts[q / (Q * Q)], x);
    xq[3 * t + 0] = x[0];
    xq[3 * t + 1] = x[1];
    xq[3 * t + 2] = x[2];
  }
}

// DOF i: trilinear map of the first element in its inverse-map list at the
// GLL node of its lattice point.
__global__ void k_dof_coords(int64_t ndof, int D1, const double* __restrict__ coords,
                             const int32_t* __restrict__ hex, const int32_t* __restrict__ off,
                             const int32_t* __restrict__ idx, const double* __restrict__ nodes,
                             double* __restrict__ out) {
  const int nd = D1 * D1 * D1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t slot = idx[off[i]];
    const int64_t e = slot / nd;
    const int k = slot % nd;
    Hex8 h;
    h.load(coords, hex, e);
    double x[3];
    h.map(nodes[k % D1], nodes[(k / D1) % D1], nodes[k / (D1 * D1)], x);
    out[3 * i + 0] = x[0];
    out[3 * i + 1] = x[1];
    out[3 * i + 2] = x[2];
  }
}

__global__ void k_mark_ess(int64_t n, int64_t ndof, const int32_t* __restrict__ ess,
                           uint8_t* __restrict__ mask, int* __restrict__ flag) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = ess[t];
    if (i < 0 || i >= ndof) {
      flag[2] = 1;
      continue;
    }
    mask[i] = 1;
  }
}

}  // namespace

fem_status fem_launch_setup(const fem_form* f, cudaStream_t s) {
  const fem_space* sp = f->space;
  if (sp->mesh->dim == 2) return fem_launch_setup_2d(f, s);
  const int64_t total = sp->ne * f->nq;
  const int grid = grid_for(total, 256);
  k_setup<<<grid, 256, 0, s>>>(sp->ne, f->q1d, f->kind, sp->mesh->d_coords, sp->mesh->d_hex, f->d_qpts,
                               f->d_qwts, f->d_coef, f->d_D, f->d_flag);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_qpoint_coords(const fem_form* f, double* xq, cudaStream_t s) {
  const fem_space* sp = f->space;
  if (sp->mesh->dim == 2) return fem_launch_qpoint_coords_2d(f, xq, s);
  const int64_t total = sp->ne * f->nq;
  k_qpoint_coords<<<grid_for(total, 256), 256, 0, s>>>(sp->ne, f->q1d, sp->mesh->d_coords, sp->mesh->d_hex,
                                                       f->d_qpts, xq);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_dof_coords(const fem_space* sp, double* out, cudaStream_t s) {
  if (sp->mesh->dim == 2) return fem_launch_dof_coords_2d(sp, out, s);
  k_dof_coords<<<grid_for(sp->ndof, 256), 256, 0, s>>>(sp->ndof, sp->D1, sp->mesh->d_coords, sp->mesh->d_hex,
                                                       sp->d_l2e_off, sp->d_l2e_idx, sp->d_nodes, out);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_mark_ess(const fem_form* f, cudaStream_t s) {
  k_mark_ess<<<grid_for(f->n_ess, 256), 256, 0, s>>>(f->n_ess, f->space->ndof, f->d_ess, f->d_ess_mask,
                                                     f->d_flag);
  FEM_LAUNCHED();
  return FEM_OK;
}

extern "C" fem_status fem_qpoint_coords(const fem_form* f, double* xq, void* stream) {
  if (!f || !xq) return fem_fail(FEM_EINVAL, "fem_qpoint_coords: NULL argument");
  return fem_launch_qpoint_coords(f, xq, (cudaStream_t)stream);
}
