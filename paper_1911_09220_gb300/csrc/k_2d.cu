// Quadrilateral (2D) counterparts of the partial-assembly kernels.
//
// Geometry (Sec. 3.1): the bilinear map of the 4 vertices on [0,1]^2, local
// vertex order (0,0), (1,0), (1,1), (0,1), or the order-k nodal map of a
// curved mesh (fem_mesh_set_nodes). Quadrature data of the 2D
// diffusion setup (Sec. 5.3): D_q = coef w_q adj(J) adj(J)^T / det J, three
// symmetric components (00, 01, 11) per point, point-major [ne][q1d^2][3];
// mass D_q = coef w_q det J, [ne][q1d^2].
//
// Action y_e = G^T B^T D B G x_e by sum factorization in two directions
// (Sec. 4.4 with d = 2), one element per row of Q threads (index t):
//   gather X[y][x] = x_L[map[y][x]]
//   S1 (y lines):  BX, GX[qx][y] = sum_x B/G[qx][x] X[y][x]
//   S2 (qx lines): grad at (qx, qy): g0 = sum_y B[qy][y] GX, g1 = sum_y G[qy][y] BX;
//                  v = D_q g; back along y: T0 = B^T_y v0, T1 = G^T_y v1
//   S3 (dy lines): Y[dy][dx] = sum_qx G[qx][dx] T0 + B[qx][dx] T1
// Every line goes through the even-odd form of its 1D operator with folded
// coefficients from constant memory (k_tables.cuh), as in 3D.
#include <type_traits>

#include "fem_internal.h"
#include "k_common.cuh"
#include "k_element.cuh"
#include "k_element2d.cuh"

namespace {

// Bilinear map of the 4 vertex coordinates; (qx, qy) index the 1D points
// pts (Gauss points for quadrature data, GLL nodes for DOF coordinates).
struct Quad4Geo {
  const double* coords;
  const int32_t* quad;
  const double* pts;
  double X[4][2];
  __device__ void load(int64_t e) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int32_t g = quad[4 * e + v];
      X[v][0] = coords[2 * (int64_t)g];
      X[v][1] = coords[2 * (int64_t)g + 1];
    }
  }
  __device__ static int cx(int v) { return v == 1 || v == 2; }
  __device__ static int cy(int v) { return v >= 2; }
  __device__ void map(int qx, int qy, double x[2]) const {
    const double a = pts[qx], b = pts[qy];
    x[0] = x[1] = 0.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double N = (cx(v) ? a : 1.0 - a) * (cy(v) ? b : 1.0 - b);
      x[0] += N * X[v][0];
      x[1] += N * X[v][1];
    }
  }
  // J[r][c] = d x_r / d xhat_c
  __device__ void jacobian(int qx, int qy, double J[2][2]) const {
    const double a = pts[qx], b = pts[qy];
    J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double fa = cx(v) ? a : 1.0 - a, da = cx(v) ? 1.0 : -1.0;
      const double fb = cy(v) ? b : 1.0 - b, db = cy(v) ? 1.0 : -1.0;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        J[r][0] += X[v][r] * da * fb;
        J[r][1] += X[v][r] * fa * db;
      }
    }
  }
};

// Order-k nodal map of the square: x(xhat) = sum_i X_i w_i(xhat) with the
// (k+1)^2 GLL Lagrange products w_i (first index fastest, in the element's
// local vertex frame) and element e's nodal coordinates X [(k+1)^2][2].
// gB, gG [npts][k+1]: the 1D functions and derivatives at the 1D points that
// (qx, qy) index.
struct NodalGeo2 {
  const double* nodes;  // [ne][(k+1)^2][2]
  const double* gB;
  const double* gG;
  int K;                // k + 1
  const double* Xe;
  __device__ void load(int64_t e) { Xe = nodes + e * (int64_t)K * K * 2; }
  __device__ void jacobian(int qx, int qy, double J[2][2]) const {
    J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.0;
    for (int i2 = 0; i2 < K; ++i2) {
      const double b2 = gB[qy * K + i2], g2 = gG[qy * K + i2];
      for (int i1 = 0; i1 < K; ++i1) {
        const double w0 = gG[qx * K + i1] * b2, w1 = gB[qx * K + i1] * g2;
        const double* x = Xe + 2 * (i2 * K + i1);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          J[r][0] += x[r] * w0;
          J[r][1] += x[r] * w1;
        }
      }
    }
  }
  __device__ void map(int qx, int qy, double xo[2]) const {
    xo[0] = xo[1] = 0.0;
    for (int i2 = 0; i2 < K; ++i2) {
      const double b2 = gB[qy * K + i2];
      for (int i1 = 0; i1 < K; ++i1) {
        const double w = gB[qx * K + i1] * b2;
        const double* x = Xe + 2 * (i2 * K + i1);
        xo[0] += x[0] * w;
        xo[1] += x[1] * w;
      }
    }
  }
};

// One thread per (element, quadrature point); q = qx + Q qy.
template <typename Geo>
__global__ void k_setup_2d(int64_t ne, int Q, int kind, Geo h, const double* __restrict__ qwts,
                           const double* __restrict__ coef, double* __restrict__ Dout, int* __restrict__ flag) {
  const int nq = Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq), qx = q % Q, qy = q / Q;
    h.load(e);
    double J[2][2];
    h.jacobian(qx, qy, J);
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (!(det > 0.0)) {
      if (atomicExch(&flag[0], 1) == 0) flag[1] = (int)e;
    }
    const double w = qwts[qx] * qwts[qy] * coef[e];
    if (kind == FEM_DIFFUSION) {
      // adj(J) = [[J11, -J01], [-J10, J00]]
      const double s = w / det;
      double* De = Dout + (e * nq + q) * 3;
      De[0] = s * (J[1][1] * J[1][1] + J[0][1] * J[0][1]);
      De[1] = -s * (J[1][1] * J[1][0] + J[0][1] * J[0][0]);
      De[2] = s * (J[1][0] * J[1][0] + J[0][0] * J[0][0]);
    } else {
      Dout[e * nq + q] = w * det;
    }
  }
}

template <typename Geo>
__global__ void k_qpoint_coords_2d(int64_t ne, int Q, Geo h, double* __restrict__ xq) {
  const int nq = Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq);
    h.load(e);
    double x[2];
    h.map(q % Q, q / Q, x);
    xq[2 * t] = x[0];
    xq[2 * t + 1] = x[1];
  }
}

// Coordinates of each DOF's GLL node, from the first element holding it
// (the geometry's 1D points are this space's GLL nodes).
template <typename Geo>
__global__ void k_dof_coords_2d(int64_t ndof, int D1, Geo h, const int32_t* __restrict__ off,
                                const int32_t* __restrict__ idx, double* __restrict__ out) {
  const int nd = D1 * D1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t slot = idx[off[i]];
    const int64_t e = slot / nd;
    const int k = slot % nd;
    h.load(e);
    double x[2];
    h.map(k % D1, k / D1, x);
    out[2 * i] = x[0];
    out[2 * i + 1] = x[1];
  }
}

// ------------------------------------------------------------ element ------
template <typename T, int D1, int Q, int NE, typename TX, bool DIFF>
__global__ void __launch_bounds__(Q * NE) k_apply_2d(const int* __restrict__ skip, int ne,
                                                     const int32_t* __restrict__ e2l, const T* __restrict__ Dq,
                                                     const TX* __restrict__ x, TX* __restrict__ ye) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int t = threadIdx.x, el = threadIdx.y;
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int nel = (int)min((int64_t)NE, ne - e0);
  quad_block<T, D1, Q, TX, DIFF>(t, el, e0, nel, e2l, Dq, sm, x, ye);
}

// Element diagonal, one thread per (element, local DOF i = ix + D1 iy):
//   diffusion  sum_q [D00 (G_qx,ix B_qy,iy)^2 + 2 D01 (G B)(B G) + D11 (B_qx,ix G_qy,iy)^2]
//   mass       sum_q D_q (B_qx,ix B_qy,iy)^2
// B, G: [Q][D1] FP64 tables in global memory.
__global__ void k_diag_2d(int64_t ne, int D1, int Q, int kind, const double* __restrict__ Dq,
                          const double* __restrict__ B, const double* __restrict__ G, double* __restrict__ ye) {
  const int nd = D1 * D1, nq = Q * Q;
  const int64_t total = ne * nd;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nd;
    const int i = (int)(t % nd), ix = i % D1, iy = i / D1;
    double acc = 0.0;
    for (int qy = 0; qy < Q; ++qy) {
      const double by = B[qy * D1 + iy], gy = G[qy * D1 + iy];
      for (int qx = 0; qx < Q; ++qx) {
        const double bx = B[qx * D1 + ix], gx = G[qx * D1 + ix];
        const int64_t q = e * nq + qx + Q * qy;
        if (kind == FEM_DIFFUSION) {
          const double a = gx * by, b = bx * gy;
          acc += Dq[q * 3] * a * a + 2.0 * Dq[q * 3 + 1] * a * b + Dq[q * 3 + 2] * b * b;
        } else {
          const double a = bx * by;
          acc += Dq[q] * a * a;
        }
      }
    }
    ye[t] = acc;
  }
}

// Load vector b_e[i] = sum_q w_q det J_q fq[e][q] phi_i(x_q), one thread per
// (element, local DOF).
template <typename Geo>
__global__ void k_rhs_2d(int64_t ne, int D1, int Q, Geo h, const double* __restrict__ qwts,
                         const double* __restrict__ B, const double* __restrict__ fq, double* __restrict__ ye) {
  const int nd = D1 * D1, nq = Q * Q;
  const int64_t total = ne * nd;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nd;
    const int i = (int)(t % nd), ix = i % D1, iy = i / D1;
    h.load(e);
    double acc = 0.0;
    for (int qy = 0; qy < Q; ++qy)
      for (int qx = 0; qx < Q; ++qx) {
        double J[2][2];
        h.jacobian(qx, qy, J);
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        acc += qwts[qx] * qwts[qy] * det * fq[e * nq + qx + Q * qy] * B[qx * D1 + ix] * B[qy * D1 + iy];
      }
    ye[t] = acc;
  }
}

// g_e = -(1/coef_e) u_e . (A_e u_e) from the element action held in ye.
__global__ void k_grad_2d(int64_t ne, int nd, const int32_t* __restrict__ e2l, const double* __restrict__ u,
                          const double* __restrict__ ye, const double* __restrict__ coef, double* __restrict__ g) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nd; ++k) s += u[e2l[e * nd + k]] * ye[e * nd + k];
    g[e] = -s / coef[e];
  }
}

template <typename T, int P, int Q, typename TX = T>
fem_status launch_apply_2d_pq(const fem_form* f, const T* D, const TX* x, TX* ye, const int* skip, cudaStream_t s) {
  constexpr int D1 = P + 1, NE = ne2(Q);
  const int ne = (int)f->space->ne;
  const size_t bytes = sizeof(T) * NE * Smem2<D1, Q>::SE;
  const dim3 block(Q, NE);
  const int grid = (ne + NE - 1) / NE;
  if (f->kind == FEM_DIFFUSION) {
    auto k = k_apply_2d<T, D1, Q, NE, TX, true>;
    if (bytes > 48 * 1024) FEM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    k<<<grid, block, bytes, s>>>(skip, ne, f->space->d_e2l, D, x, ye);
  } else {
    auto k = k_apply_2d<T, D1, Q, NE, TX, false>;
    if (bytes > 48 * 1024) FEM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    k<<<grid, block, bytes, s>>>(skip, ne, f->space->d_e2l, D, x, ye);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

}  // namespace

fem_status fem_2d_tables_init() { return fem_tables_ensure(); }

fem_status fem_launch_setup_2d(const fem_form* f, cudaStream_t s) {
  const fem_space* sp = f->space;
  const fem_mesh* m = sp->mesh;
  const int grid = grid_for(sp->ne * f->nq, 256);
  if (m->geo_k > 0) {
    FEM_TRY(fem_form_geo_tables(f));
    const NodalGeo2 g{m->d_gnodes, f->d_gB, f->d_gG, m->geo_k + 1, nullptr};
    k_setup_2d<NodalGeo2><<<grid, 256, 0, s>>>(sp->ne, f->q1d, f->kind, g, f->d_qwts, f->d_coef, f->d_D, f->d_flag);
  } else {
    const Quad4Geo g{m->d_coords, m->d_hex, f->d_qpts, {}};
    k_setup_2d<Quad4Geo><<<grid, 256, 0, s>>>(sp->ne, f->q1d, f->kind, g, f->d_qwts, f->d_coef, f->d_D, f->d_flag);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_qpoint_coords_2d(const fem_form* f, double* xq, cudaStream_t s) {
  const fem_space* sp = f->space;
  const fem_mesh* m = sp->mesh;
  const int grid = grid_for(sp->ne * f->nq, 256);
  if (m->geo_k > 0) {
    FEM_TRY(fem_form_geo_tables(f));
    const NodalGeo2 g{m->d_gnodes, f->d_gB, f->d_gG, m->geo_k + 1, nullptr};
    k_qpoint_coords_2d<NodalGeo2><<<grid, 256, 0, s>>>(sp->ne, f->q1d, g, xq);
  } else {
    const Quad4Geo g{m->d_coords, m->d_hex, f->d_qpts, {}};
    k_qpoint_coords_2d<Quad4Geo><<<grid, 256, 0, s>>>(sp->ne, f->q1d, g, xq);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_dof_coords_2d(const fem_space* sp, double* out, cudaStream_t s) {
  const fem_mesh* m = sp->mesh;
  const int grid = grid_for(sp->ndof, 256);
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
    const NodalGeo2 g{m->d_gnodes, sp->d_gBn, sp->d_gBn, m->geo_k + 1, nullptr};
    k_dof_coords_2d<NodalGeo2><<<grid, 256, 0, s>>>(sp->ndof, sp->D1, g, sp->d_l2e_off, sp->d_l2e_idx, out);
  } else {
    const Quad4Geo g{m->d_coords, m->d_hex, sp->d_nodes, {}};
    k_dof_coords_2d<Quad4Geo><<<grid, 256, 0, s>>>(sp->ndof, sp->D1, g, sp->d_l2e_off, sp->d_l2e_idx, out);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_apply_element_2d(const fem_form* f, int dtype, const void* x, void* ye, cudaStream_t s,
                                       const int* skip) {
  const int p = f->space->p, q = f->q1d;
  if (dtype == FEM_F64) {
#define X(P, Q) \
  if (p == P && q == Q) return launch_apply_2d_pq<double, P, Q>(f, f->d_D, (const double*)x, (double*)ye, skip, s);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else if (dtype == FEM_F32) {
    FEM_TRY(fem_form_ensure_f32(f, s));
#define X(P, Q) \
  if (p == P && q == Q) return launch_apply_2d_pq<float, P, Q>(f, f->d_D32, (const float*)x, (float*)ye, skip, s);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else if (dtype == FEM_DF64) {
    FEM_TRY(fem_form_ensure_df64(f, s));
    const df64* D = reinterpret_cast<const df64*>(f->d_Ddf);
#define X(P, Q) \
  if (p == P && q == Q) return launch_apply_2d_pq<df64, P, Q, double>(f, D, (const double*)x, (double*)ye, skip, s);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else {
    return fem_fail(FEM_EINVAL, "apply: unknown dtype %d", dtype);
  }
  return fem_fail(FEM_EUNSUPPORTED, "apply: (p=%d, q1d=%d) not compiled", p, q);
}

fem_status fem_launch_diag_element_2d(const fem_form* f, double* ye, cudaStream_t s) {
  const fem_space* sp = f->space;
  k_diag_2d<<<grid_for(sp->ne * sp->nd, 256), 256, 0, s>>>(sp->ne, sp->D1, f->q1d, f->kind, f->d_D, f->d_B, f->d_G,
                                                           ye);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_rhs_element_2d(const fem_form* f, const double* fq, double* ye, cudaStream_t s) {
  const fem_space* sp = f->space;
  const fem_mesh* m = sp->mesh;
  const int grid = grid_for(sp->ne * sp->nd, 256);
  if (m->geo_k > 0) {
    FEM_TRY(fem_form_geo_tables(f));
    const NodalGeo2 g{m->d_gnodes, f->d_gB, f->d_gG, m->geo_k + 1, nullptr};
    k_rhs_2d<NodalGeo2><<<grid, 256, 0, s>>>(sp->ne, sp->D1, f->q1d, g, f->d_qwts, f->d_B, fq, ye);
  } else {
    const Quad4Geo g{m->d_coords, m->d_hex, f->d_qpts, {}};
    k_rhs_2d<Quad4Geo><<<grid, 256, 0, s>>>(sp->ne, sp->D1, f->q1d, g, f->d_qwts, f->d_B, fq, ye);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_grad_2d(const fem_form* f, const double* u, double* g, cudaStream_t s) {
  const fem_space* sp = f->space;
  double* ye = (double*)f->d_ye;
  FEM_TRY(fem_launch_apply_element_2d(f, FEM_F64, u, ye, s, nullptr));
  k_grad_2d<<<grid_for(sp->ne, 256), 256, 0, s>>>(sp->ne, sp->nd, sp->d_e2l, u, ye, f->d_coef, g);
  FEM_LAUNCHED();
  return FEM_OK;
}
