// Partial-assembly setup: quadrature data D at every element and Gauss point
// (Sec. 4.3, "setup phase that evaluates and stores D"), plus coordinate
// helpers (quadrature points, DOF nodes) and the essential-DOF mask.
#include "fem_internal.h"
#include "k_common.cuh"
#include "k_geom.cuh"

namespace {

// One thread per (element, quadrature point).
//   diffusion: D = coef * w * adj(J) adj(J)^T / det J  (= coef w det J J^-1 J^-T),
//              components 00,01,02,11,12,22;
//   mass:      D = coef * w * det J.
// Geo: Hex8Geo (vertex geometry) or NodalGeo (order-k nodal geometry).
template <typename Geo>
__global__ void k_setup(int64_t ne, int Q, int kind, Geo geo, const double* __restrict__ qwts,
                        const double* __restrict__ coef, double* __restrict__ Dout, int* __restrict__ flag) {
  const int nq = Q * Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq);
    const int q1 = q % Q, q2 = (q / Q) % Q, q3 = q / (Q * Q);
    Geo h = geo;
    h.load(e);
    double J[3][3];
    h.jacobian(q1, q2, q3, J);
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

// Convection: D = coef * w * adj(J) beta (= coef w det J J^-1 beta),
// point-major [e][q][3]; beta [e][q][3] physical.
template <typename Geo>
__global__ void k_setup_conv(int64_t ne, int Q, Geo geo, const double* __restrict__ qwts,
                             const double* __restrict__ coef, const double* __restrict__ beta,
                             double* __restrict__ Dout, int* __restrict__ flag) {
  const int nq = Q * Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq);
    const int q1 = q % Q, q2 = (q / Q) % Q, q3 = q / (Q * Q);
    Geo h = geo;
    h.load(e);
    double J[3][3];
    h.jacobian(q1, q2, q3, J);
    double C[3][3];  // cofactors; adj(J)[a][b] = C[b][a]
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
    const double* b = beta + t * 3;
    double* De = Dout + t * 3;
#pragma unroll
    for (int a = 0; a < 3; ++a) De[a] = w * (C[0][a] * b[0] + C[1][a] * b[1] + C[2][a] * b[2]);
  }
}

// Elasticity: per point J^-1 (row-major, [3 s + r] = d xhat_s / d x_r =
// adj(J)[s][r] / det J), w det J lambda_e, w det J mu_e and a zero pad
// (12 values, point-major [e][q][12]: 16-byte aligned records for the
// apply's vector loads).
template <typename Geo>
__global__ void k_setup_elast(int64_t ne, int Q, Geo geo, const double* __restrict__ qwts,
                              const double* __restrict__ lam, const double* __restrict__ mu,
                              double* __restrict__ Dout, int* __restrict__ flag) {
  const int nq = Q * Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq);
    const int q1 = q % Q, q2 = (q / Q) % Q, q3 = q / (Q * Q);
    Geo h = geo;
    h.load(e);
    double J[3][3];
    h.jacobian(q1, q2, q3, J);
    double C[3][3];  // cofactors; adj(J)[a][b] = C[b][a]
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
    const double wd = qwts[q1] * qwts[q2] * qwts[q3] * det;
    double* De = Dout + t * 12;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < 3; ++r) De[3 * a + r] = C[r][a] / det;
    De[9] = wd * lam[e];
    De[10] = wd * mu[e];
    De[11] = 0.0;
  }
}

// Elasticity diagonal: the symmetric matrix of component c at every point,
//   D^c = w det J ((lambda + mu) a_c a_c^T + mu J^-1 J^-T),  a_c[s] = J^-1[s][c],
// in the diffusion layout [e][q][6] (00, 01, 02, 11, 12, 22): the (c, c)
// block's diagonal is then the diffusion diagonal with D^c.
__global__ void k_elast_diag_D(int64_t total, int c, const double* __restrict__ De, double* __restrict__ Dc) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double* m = De + t * 12;
    const double lm = m[9] + m[10], mu = m[10];
    double* o = Dc + t * 6;
    const int S[6] = {0, 0, 0, 1, 1, 2}, U[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double* ms = m + 3 * S[k];
      const double* mt = m + 3 * U[k];
      o[k] = lm * ms[c] * mt[c] + mu * (ms[0] * mt[0] + ms[1] * mt[1] + ms[2] * mt[2]);
    }
  }
}

// x at the tensor points (q1, q2, q3) of a P^3 set: the Gauss points
// (quadrature-point coordinates, out [ne][P^3][3]).
template <typename Geo>
__global__ void k_qpoint_coords(int64_t ne, int P, Geo geo, double* __restrict__ xq) {
  const int np = P * P * P;
  const int64_t total = ne * np;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / np;
    const int q = (int)(t % np);
    Geo h = geo;
    h.load(e);
    double x[3];
    h.map(q % P, (q / P) % P, q / (P * P), x);
    xq[3 * t + 0] = x[0];
    xq[3 * t + 1] = x[1];
    xq[3 * t + 2] = x[2];
  }
}

// DOF i: the map of the first element in its inverse-map list at the GLL
// node of its lattice point (geo's point set = the space's GLL nodes).
template <typename Geo>
__global__ void k_dof_coords(int64_t ndof, int D1, Geo geo, const int32_t* __restrict__ off,
                             const int32_t* __restrict__ idx, double* __restrict__ out) {
  const int nd = D1 * D1 * D1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t slot = idx[off[i]];
    const int64_t e = slot / nd;
    const int k = slot % nd;
    Geo h = geo;
    h.load(e);
    double x[3];
    h.map(k % D1, (k / D1) % D1, k / (D1 * D1), x);
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
  const fem_mesh* m = sp->mesh;
  const bool conv = f->kind == FEM_CONVECTION, elast = f->kind == FEM_ELASTICITY;
  if (m->geo_k > 0) {
    FEM_TRY(fem_form_geo_tables(f));
    const NodalGeo g{m->d_gnodes, f->d_gB, f->d_gG, m->geo_k + 1, nullptr};
    if (elast)
      k_setup_elast<NodalGeo><<<grid, 256, 0, s>>>(sp->ne, f->q1d, g, f->d_qwts, f->d_coef, f->d_mu, f->d_D,
                                                   f->d_flag);
    else if (conv)
      k_setup_conv<NodalGeo><<<grid, 256, 0, s>>>(sp->ne, f->q1d, g, f->d_qwts, f->d_coef, f->d_beta, f->d_D,
                                                  f->d_flag);
    else
      k_setup<NodalGeo><<<grid, 256, 0, s>>>(sp->ne, f->q1d, f->kind, g, f->d_qwts, f->d_coef, f->d_D, f->d_flag);
  } else {
    const Hex8Geo g{m->d_coords, m->d_hex, f->d_qpts, {}};
    if (elast)
      k_setup_elast<Hex8Geo><<<grid, 256, 0, s>>>(sp->ne, f->q1d, g, f->d_qwts, f->d_coef, f->d_mu, f->d_D,
                                                  f->d_flag);
    else if (conv)
      k_setup_conv<Hex8Geo><<<grid, 256, 0, s>>>(sp->ne, f->q1d, g, f->d_qwts, f->d_coef, f->d_beta, f->d_D,
                                                 f->d_flag);
    else
      k_setup<Hex8Geo><<<grid, 256, 0, s>>>(sp->ne, f->q1d, f->kind, g, f->d_qwts, f->d_coef, f->d_D, f->d_flag);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_qpoint_coords(const fem_form* f, double* xq, cudaStream_t s) {
  const fem_space* sp = f->space;
  if (sp->mesh->dim == 2) return fem_launch_qpoint_coords_2d(f, xq, s);
  const int64_t total = sp->ne * f->nq;
  const fem_mesh* m = sp->mesh;
  if (m->geo_k > 0) {
    FEM_TRY(fem_form_geo_tables(f));
    const NodalGeo g{m->d_gnodes, f->d_gB, f->d_gG, m->geo_k + 1, nullptr};
    k_qpoint_coords<NodalGeo><<<grid_for(total, 256), 256, 0, s>>>(sp->ne, f->q1d, g, xq);
  } else {
    const Hex8Geo g{m->d_coords, m->d_hex, f->d_qpts, {}};
    k_qpoint_coords<Hex8Geo><<<grid_for(total, 256), 256, 0, s>>>(sp->ne, f->q1d, g, xq);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_dof_coords(const fem_space* sp, double* out, cudaStream_t s) {
  if (sp->mesh->dim == 2) return fem_launch_dof_coords_2d(sp, out, s);
  const fem_mesh* m = sp->mesh;
  if (m->geo_k > 0) {
    // order-k geometry functions at this space's GLL nodes, [D1][k+1]
    fem_space* spm = const_cast<fem_space*>(sp);
    if (spm->gBn_k != m->geo_k) {
      std::vector<double> nk, B, G;
      fem_gll_nodes(m->geo_k, nk);
      fem_lagrange_tables(nk, sp->nodes, B, G);
      dev_free(spm->d_gBn);
      FEM_TRY(dev_alloc(&spm->d_gBn, B.size()));
      FEM_CUDA(cudaMemcpy(spm->d_gBn, B.data(), sizeof(double) * B.size(), cudaMemcpyHostToDevice));
      spm->gBn_k = m->geo_k;
    }
    const NodalGeo g{m->d_gnodes, sp->d_gBn, sp->d_gBn, m->geo_k + 1, nullptr};
    k_dof_coords<NodalGeo><<<grid_for(sp->ndof, 256), 256, 0, s>>>(sp->ndof, sp->D1, g, sp->d_l2e_off,
                                                                   sp->d_l2e_idx, out);
  } else {
    const Hex8Geo g{m->d_coords, m->d_hex, sp->d_nodes, {}};
    k_dof_coords<Hex8Geo><<<grid_for(sp->ndof, 256), 256, 0, s>>>(sp->ndof, sp->D1, g, sp->d_l2e_off,
                                                                  sp->d_l2e_idx, out);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_mark_ess(const fem_form* f, cudaStream_t s) {
  k_mark_ess<<<grid_for(f->n_ess, 256), 256, 0, s>>>(f->n_ess, fem_form_len(f), f->d_ess, f->d_ess_mask,
                                                     f->d_flag);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_elasticity_diag_D(const fem_form* f, int c, double* Dc, cudaStream_t s) {
  const int64_t total = f->space->ne * f->nq;
  k_elast_diag_D<<<grid_for(total, 256), 256, 0, s>>>(total, c, f->d_D, Dc);
  FEM_LAUNCHED();
  return FEM_OK;
}

extern "C" fem_status fem_qpoint_coords(const fem_form* f, double* xq, void* stream) {
  if (!f || !xq) return fem_fail(FEM_EINVAL, "fem_qpoint_coords: NULL argument");
  return fem_launch_qpoint_coords(f, xq, (cudaStream_t)stream);
}
