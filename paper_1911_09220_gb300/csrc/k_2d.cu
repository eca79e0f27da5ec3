// Quadrilateral (2D) counterparts of the partial-assembly kernels.
//
// Geometry: bilinear map of the 4 vertices on [0,1]^2 (Sec. 3.1), local
// vertex order (0,0), (1,0), (1,1), (0,1). Quadrature data of the 2D
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

namespace {

struct Quad4 {
  double X[4][2];
  __device__ void load(const double* __restrict__ coords, const int32_t* __restrict__ quad, int64_t e) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int32_t g = quad[4 * e + v];
      X[v][0] = coords[2 * (int64_t)g];
      X[v][1] = coords[2 * (int64_t)g + 1];
    }
  }
  __device__ static int cx(int v) { return v == 1 || v == 2; }
  __device__ static int cy(int v) { return v >= 2; }
  __device__ void map(double a, double b, double x[2]) const {
    x[0] = x[1] = 0.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const double N = (cx(v) ? a : 1.0 - a) * (cy(v) ? b : 1.0 - b);
      x[0] += N * X[v][0];
      x[1] += N * X[v][1];
    }
  }
  // J[r][c] = d x_r / d xhat_c
  __device__ void jacobian(double a, double b, double J[2][2]) const {
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

// One thread per (element, quadrature point); q = qx + Q qy.
__global__ void k_setup_2d(int64_t ne, int Q, int kind, const double* __restrict__ coords,
                           const int32_t* __restrict__ quad, const double* __restrict__ qpts,
                           const double* __restrict__ qwts, const double* __restrict__ coef,
                           double* __restrict__ Dout, int* __restrict__ flag) {
  const int nq = Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq), qx = q % Q, qy = q / Q;
    Quad4 h;
    h.load(coords, quad, e);
    double J[2][2];
    h.jacobian(qpts[qx], qpts[qy], J);
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

__global__ void k_qpoint_coords_2d(int64_t ne, int Q, const double* __restrict__ coords,
                                   const int32_t* __restrict__ quad, const double* __restrict__ qpts,
                                   double* __restrict__ xq) {
  const int nq = Q * Q;
  const int64_t total = ne * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nq;
    const int q = (int)(t % nq);
    Quad4 h;
    h.load(coords, quad, e);
    double x[2];
    h.map(qpts[q % Q], qpts[q / Q], x);
    xq[2 * t] = x[0];
    xq[2 * t + 1] = x[1];
  }
}

__global__ void k_dof_coords_2d(int64_t ndof, int D1, const double* __restrict__ coords,
                                const int32_t* __restrict__ quad, const int32_t* __restrict__ off,
                                const int32_t* __restrict__ idx, const double* __restrict__ nodes,
                                double* __restrict__ out) {
  const int nd = D1 * D1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t slot = idx[off[i]];
    const int64_t e = slot / nd;
    const int k = slot % nd;
    Quad4 h;
    h.load(coords, quad, e);
    double x[2];
    h.map(nodes[k % D1], nodes[k / D1], x);
    out[2 * i] = x[0];
    out[2 * i + 1] = x[1];
  }
}

// ------------------------------------------------------------ element ------
template <int D1, int Q>
struct Smem2 {
  static constexpr int XP = D1 | 1;  // padded x rows of X
  static constexpr int YP = D1 | 1;  // padded y rows of BX, GX
  static constexpr int QP = Q | 1;   // padded qx rows of T0, T1
  static constexpr int SE = D1 * XP + 2 * Q * YP + 2 * D1 * QP;  // per element, in T
};

// Elements per block: rows of Q threads, about 128 threads per block.
__host__ __device__ constexpr int ne2(int Q) { return Q <= 3 ? 42 : Q <= 4 ? 32 : Q <= 6 ? 21 : Q <= 8 ? 16 : 12; }

template <typename T, int D1, int Q, int NE, typename TX, bool DIFF>
__global__ void __launch_bounds__(Q * NE) k_apply_2d(const int* __restrict__ skip, int ne,
                                                     const int32_t* __restrict__ e2l, const T* __restrict__ Dq,
                                                     const TX* __restrict__ x, TX* __restrict__ ye) {
  if (skip && *skip) return;
  using L = Smem2<D1, Q>;
  constexpr int XP = L::XP, YP = L::YP, QP = L::QP, ND = D1 * D1, NQ = Q * Q;
  constexpr int BF = eo_off(D1, Q, 0), GF = eo_off(D1, Q, 1), BT = eo_off(D1, Q, 2), GT = eo_off(D1, Q, 3);
  // slab offsets: X [y][XP], BX, GX [qx][YP], T0, T1 [dy][QP]
  constexpr int OBX = D1 * XP, OGX = OBX + Q * YP, OT0 = OGX + Q * YP, OT1 = OT0 + D1 * QP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int t = threadIdx.x, el = threadIdx.y, tid = t + Q * el;
  const int64_t e0 = (int64_t)blockIdx.x * NE, e = e0 + el;
  const int nel = (int)min((int64_t)NE, ne - e0);
  const bool valid = e < ne;
  if (valid) {
    T* sX = sm + el * L::SE;
    const int32_t* map = e2l + e * ND;
    for (int k = t; k < ND; k += Q) sX[(k / D1) * XP + k % D1] = fe_from<T>(__ldg(x + __ldg(map + k)));
  }
  __syncthreads();
  // S1 and S3 have D1 lines per element: the lines of all nel elements are
  // packed onto the lowest thread ids (full warps); S2 has Q lines per
  // element and keeps one row of Q threads per element.
  if (tid < nel * D1) {  // S1: line y along x
    T* s = sm + (tid / D1) * L::SE;
    const int t = tid % D1;
    T *sX = s, *sBX = s + OBX, *sGX = s + OGX;
    T xr[D1], bx[Q], gx[Q];
#pragma unroll
    for (int d = 0; d < D1; ++d) xr[d] = sX[t * XP + d];
    if constexpr (DIFF) {
      T ev[(D1 + 1) / 2], od[D1 / 2 > 0 ? D1 / 2 : 1];
      eo_split<T, D1>(xr, ev, od);
      eo_apply<T, Q, D1, 1, BF>(ev, od, bx);
      eo_apply<T, Q, D1, -1, GF>(ev, od, gx);
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) {
        sBX[qx * YP + t] = bx[qx];
        sGX[qx * YP + t] = gx[qx];
      }
    } else {
      eo_line<T, Q, D1, 1, BF>(xr, bx);
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) sBX[qx * YP + t] = bx[qx];
    }
  }
  __syncthreads();
  {  // S2: line qx along y, D at every point, back along y (t < Q always)
    const int qx = t;
    T* s = sm + el * L::SE;
    T *sBX = s + OBX, *sGX = s + OGX, *sT0 = s + OT0, *sT1 = s + OT1;
    T br[D1], t0[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) br[d] = sBX[qx * YP + d];
    if constexpr (DIFF) {
      T gr[D1], g0[Q], g1[Q], t1[D1];
#pragma unroll
      for (int d = 0; d < D1; ++d) gr[d] = sGX[qx * YP + d];
      eo_line<T, Q, D1, 1, BF>(gr, g0);   // d/dx
      eo_line<T, Q, D1, -1, GF>(br, g1);  // d/dy
      const T* Dp = Dq + ((size_t)e * NQ + qx) * 3;
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) {
        T d00 = 0, d01 = 0, d11 = 0;
        if (valid) {
          d00 = fe_ldg(Dp + qy * Q * 3);
          d01 = fe_ldg(Dp + qy * Q * 3 + 1);
          d11 = fe_ldg(Dp + qy * Q * 3 + 2);
        }
        const T a0 = g0[qy], a1 = g1[qy];
        g0[qy] = fe_norm(d00 * a0 + d01 * a1);
        g1[qy] = fe_norm(d01 * a0 + d11 * a1);
      }
      eo_line<T, D1, Q, 1, BT>(g0, t0);
      eo_line<T, D1, Q, -1, GT>(g1, t1);
#pragma unroll
      for (int dy = 0; dy < D1; ++dy) {
        sT0[dy * QP + qx] = t0[dy];
        sT1[dy * QP + qx] = t1[dy];
      }
    } else {
      T u[Q];
      eo_line<T, Q, D1, 1, BF>(br, u);
      const T* Dp = Dq + (size_t)e * NQ + qx;
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) u[qy] = valid ? fe_norm(fe_ldg(Dp + qy * Q) * u[qy]) : T(0);
      eo_line<T, D1, Q, 1, BT>(u, t0);
#pragma unroll
      for (int dy = 0; dy < D1; ++dy) sT0[dy * QP + qx] = t0[dy];
    }
  }
  __syncthreads();
  if (tid < nel * D1) {  // S3: line dy along qx
    const int el3 = tid / D1, t = tid % D1;
    T* s = sm + el3 * L::SE;
    const T *sT0 = s + OT0, *sT1 = s + OT1;
    T a0[Q], y1[D1];
#pragma unroll
    for (int q = 0; q < Q; ++q) a0[q] = sT0[t * QP + q];
    TX* out = ye + (e0 + el3) * ND + t * D1;
    if constexpr (DIFF) {
      T a1[Q], y2[D1];
#pragma unroll
      for (int q = 0; q < Q; ++q) a1[q] = sT1[t * QP + q];
      eo_line<T, D1, Q, -1, GT>(a0, y1);
      eo_line<T, D1, Q, 1, BT>(a1, y2);
#pragma unroll
      for (int dx = 0; dx < D1; ++dx) fe_store(out + dx, y1[dx] + y2[dx]);
    } else {
      eo_line<T, D1, Q, 1, BT>(a0, y1);
#pragma unroll
      for (int dx = 0; dx < D1; ++dx) fe_store(out + dx, y1[dx]);
    }
  }
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
__global__ void k_rhs_2d(int64_t ne, int D1, int Q, const double* __restrict__ coords,
                         const int32_t* __restrict__ quad, const double* __restrict__ qpts,
                         const double* __restrict__ qwts, const double* __restrict__ B, const double* __restrict__ fq,
                         double* __restrict__ ye) {
  const int nd = D1 * D1, nq = Q * Q;
  const int64_t total = ne * nd;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nd;
    const int i = (int)(t % nd), ix = i % D1, iy = i / D1;
    Quad4 h;
    h.load(coords, quad, e);
    double acc = 0.0;
    for (int qy = 0; qy < Q; ++qy)
      for (int qx = 0; qx < Q; ++qx) {
        double J[2][2];
        h.jacobian(qpts[qx], qpts[qy], J);
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
  k_setup_2d<<<grid_for(sp->ne * f->nq, 256), 256, 0, s>>>(sp->ne, f->q1d, f->kind, sp->mesh->d_coords,
                                                           sp->mesh->d_hex, f->d_qpts, f->d_qwts, f->d_coef,
                                                           f->d_D, f->d_flag);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_qpoint_coords_2d(const fem_form* f, double* xq, cudaStream_t s) {
  const fem_space* sp = f->space;
  k_qpoint_coords_2d<<<grid_for(sp->ne * f->nq, 256), 256, 0, s>>>(sp->ne, f->q1d, sp->mesh->d_coords,
                                                                   sp->mesh->d_hex, f->d_qpts, xq);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_dof_coords_2d(const fem_space* sp, double* out, cudaStream_t s) {
  k_dof_coords_2d<<<grid_for(sp->ndof, 256), 256, 0, s>>>(sp->ndof, sp->D1, sp->mesh->d_coords, sp->mesh->d_hex,
                                                          sp->d_l2e_off, sp->d_l2e_idx, sp->d_nodes, out);
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
  k_rhs_2d<<<grid_for(sp->ne * sp->nd, 256), 256, 0, s>>>(sp->ne, sp->D1, f->q1d, sp->mesh->d_coords,
                                                          sp->mesh->d_hex, f->d_qpts, f->d_qwts, f->d_B, fq, ye);
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
