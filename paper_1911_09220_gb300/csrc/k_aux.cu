// Assembled diagonal, load vector, compliance gradient and right-hand-side
// lifting, all by sum factorization over the same (Q x Q) thread planes as the
// apply kernels, followed by the atomic-free inverse-map scatter.
#include "fem_internal.h"
#include "k_common.cuh"
#include "k_geom.cuh"

namespace {

constexpr int ne_per_block_aux(int p) { return p <= 2 ? 8 : p <= 4 ? 4 : 2; }

// 1D factor of a squared basis product: kind 0 = B*B, 1 = G*G, 2 = G*B.
__device__ __forceinline__ double sq(const double* sB, const double* sG, int kind, int i) {
  return kind == 0 ? sB[i] * sB[i] : kind == 1 ? sG[i] * sG[i] : sG[i] * sB[i];
}

// Diagonal of the element operator (needed for Jacobi: with PA no matrix
// entries exist, Sec. 4.4 / Sec. 5.2):
//   diag_e[i] = sum_q sum_ab D_ab(q) dphi_i/dxhat_a(q) dphi_i/dxhat_b(q).
// With phi_i = l_i1(x) l_i2(y) l_i3(z), each (a,b) term factorises into
// products of squared 1D tables, e.g. D_01 -> (G.B)_x (B.G)_y (B.B)_z, so
// each component is one transposed sum-factorized contraction.
template <int D1, int Q, int NE>
__global__ void __launch_bounds__(Q * Q * NE)
k_diag(int ne, int kind, const double* __restrict__ Dq, const double* __restrict__ Bg,
       const double* __restrict__ Gg, double* __restrict__ ye) {
  constexpr int ND = D1 * D1 * D1, NQ = Q * Q * Q;
  constexpr int SE = D1 * Q * Q + 3 * D1 * D1 * Q;
  __shared__ double sB[Q * D1], sG[Q * D1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + Q * (ty + Q * tz);
  for (int i = tid; i < Q * D1; i += Q * Q * NE) {
    sB[i] = Bg[i];
    sG[i] = Gg[i];
  }
  const int e = blockIdx.x * NE + tz;
  const bool valid = e < ne;
  double* sA = sm + tz * SE;             // [dz][qy][qx]
  double* sC = sA + D1 * Q * Q;          // 3 classes x [dz][dy][qx]
  for (int i = tx + Q * ty; i < 3 * D1 * D1 * Q; i += Q * Q) sC[i] = 0.0;
  // components: (x kind, y kind, z kind, factor); the x kind is the class
  const int ncomp = kind == FEM_DIFFUSION ? 6 : 1;
  const int KX[6] = {1, 2, 2, 0, 0, 0}, KY[6] = {0, 2, 0, 1, 2, 0}, KZ[6] = {0, 0, 2, 0, 2, 1};
  const double FAC[6] = {1, 2, 2, 1, 2, 1};
  __syncthreads();
  for (int c = 0; c < ncomp; ++c) {
    const int kx = kind == FEM_DIFFUSION ? KX[c] : 0, ky = kind == FEM_DIFFUSION ? KY[c] : 0,
              kz = kind == FEM_DIFFUSION ? KZ[c] : 0;
    const double fac = kind == FEM_DIFFUSION ? FAC[c] : 1.0;
    double a[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) a[d] = 0.0;
    if (valid) {
      // point-major D: component c of point q at (e * NQ + q) * ncomp + c
      const double* De = Dq + ((size_t)e * NQ + ty * Q + tx) * ncomp + c;
      for (int qz = 0; qz < Q; ++qz) {
        const double v = fac * De[(size_t)qz * Q * Q * ncomp];
#pragma unroll
        for (int d = 0; d < D1; ++d) a[d] += sq(sB, sG, kz, qz * D1 + d) * v;
      }
    }
#pragma unroll
    for (int d = 0; d < D1; ++d) sA[(d * Q + ty) * Q + tx] = a[d];
    __syncthreads();
    if (ty < D1) {  // y contraction, accumulated into the class of the x factor
      double* out = sC + kx * D1 * D1 * Q;
      for (int dz = 0; dz < D1; ++dz) {
        double acc = 0.0;
        for (int qy = 0; qy < Q; ++qy) acc += sq(sB, sG, ky, qy * D1 + ty) * sA[(dz * Q + qy) * Q + tx];
        out[(dz * D1 + ty) * Q + tx] += acc;
      }
    }
    __syncthreads();
  }
  if (valid && tx < D1 && ty < D1) {
    for (int dz = 0; dz < D1; ++dz) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int qx = 0; qx < Q; ++qx)
          acc += sq(sB, sG, k, qx * D1 + tx) * sC[k * D1 * D1 * Q + (dz * D1 + ty) * Q + qx];
      ye[(size_t)e * ND + (dz * D1 + ty) * D1 + tx] = acc;
    }
  }
}

// Trilinear Jacobian determinant at reference point (a, b, c) from the 8
// corner coordinates X[v][d] (Sec. 3.1, Eq. mesh_eq_x).
__device__ double hex_detj(const double* X, double a, double b, double c) {
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int v = 0; v < 8; ++v) {
    const int cx = (v == 1 || v == 2 || v == 5 || v == 6), cy = (v == 2 || v == 3 || v == 6 || v == 7),
              cz = v >= 4;
    const double fa = cx ? a : 1 - a, fb = cy ? b : 1 - b, fc = cz ? c : 1 - c;
    const double g0 = (cx ? 1 : -1) * fb * fc, g1 = fa * (cy ? 1 : -1) * fc, g2 = fa * fb * (cz ? 1 : -1);
    for (int r = 0; r < 3; ++r) {
      J[r][0] += X[3 * v + r] * g0;
      J[r][1] += X[3 * v + r] * g1;
      J[r][2] += X[3 * v + r] * g2;
    }
  }
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// Element load vectors b_e[i] = sum_q w_q detJ_q fq(e,q) phi_i(q)
// (Sec. 2, b_i = int f phi_i): B^T B^T B^T applied to the weighted values.
template <int D1, int Q, int NE>
__global__ void __launch_bounds__(Q * Q * NE)
k_rhs(int ne, const double* __restrict__ coords, const int32_t* __restrict__ hex,
      const double* __restrict__ qpts, const double* __restrict__ qwts, const double* __restrict__ Bg,
      const double* __restrict__ fq, double* __restrict__ ye, NodalGeo ng) {
  constexpr int ND = D1 * D1 * D1, NQ = Q * Q * Q;
  constexpr int SE = D1 * Q * Q + D1 * D1 * Q + 24;
  __shared__ double sB[Q * D1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + Q * (ty + Q * tz);
  for (int i = tid; i < Q * D1; i += Q * Q * NE) sB[i] = Bg[i];
  const int e = blockIdx.x * NE + tz;
  const bool valid = e < ne;
  double* sT = sm + tz * SE;
  double* sU = sT + D1 * Q * Q;
  double* sX = sU + D1 * D1 * Q;
  const int lt = tx + Q * ty;
  if (valid)
    for (int i = lt; i < 24; i += Q * Q) sX[i] = coords[3 * (int64_t)hex[8 * (int64_t)e + i / 3] + i % 3];
  __syncthreads();
  double t[D1];
#pragma unroll
  for (int d = 0; d < D1; ++d) t[d] = 0.0;
  if (valid) {
    NodalGeo g = ng;  // ng.K > 0: curved mesh, det J from the nodal map
    if (g.K > 0) g.load(e);
    for (int qz = 0; qz < Q; ++qz) {
      double dj;
      if (g.K > 0) {
        double J[3][3];
        g.jacobian(tx, ty, qz, J);
        dj = det3(J);
      } else {
        dj = hex_detj(sX, qpts[tx], qpts[ty], qpts[qz]);
      }
      const double v = qwts[tx] * qwts[ty] * qwts[qz] * dj * fq[(size_t)e * NQ + (qz * Q + ty) * Q + tx];
#pragma unroll
      for (int d = 0; d < D1; ++d) t[d] += sB[qz * D1 + d] * v;
    }
  }
#pragma unroll
  for (int d = 0; d < D1; ++d) sT[(d * Q + ty) * Q + tx] = t[d];
  __syncthreads();
  if (ty < D1) {
    for (int dz = 0; dz < D1; ++dz) {
      double a = 0.0;
      for (int q = 0; q < Q; ++q) a += sB[q * D1 + ty] * sT[(dz * Q + q) * Q + tx];
      sU[(dz * D1 + ty) * Q + tx] = a;
    }
  }
  __syncthreads();
  if (valid && tx < D1 && ty < D1) {
    for (int dz = 0; dz < D1; ++dz) {
      double a = 0.0;
      for (int q = 0; q < Q; ++q) a += sB[q * D1 + tx] * sU[(dz * D1 + ty) * Q + q];
      ye[(size_t)e * ND + (dz * D1 + ty) * D1 + tx] = a;
    }
  }
}

// Compliance gradient g_e = -(1/coef_e) sum_q gradhat(u)^T D_q gradhat(u)
// (= -u_e^T Khat_e u_e): the forward half of the diffusion apply, the
// quadratic form at each point, and a fixed-order reduction per element.
template <int D1, int Q, int NE>
__global__ void __launch_bounds__(Q * Q * NE)
k_grad(int ne, const int32_t* __restrict__ e2l, const double* __restrict__ Dq,
       const double* __restrict__ coef, const double* __restrict__ Bg, const double* __restrict__ Gg,
       const double* __restrict__ u, double* __restrict__ g) {
  constexpr int ND = D1 * D1 * D1, NQ = Q * Q * Q;
  constexpr int SE = ND + 2 * D1 * D1 * Q + Q * Q;
  __shared__ double sB[Q * D1], sG[Q * D1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + Q * (ty + Q * tz);
  for (int i = tid; i < Q * D1; i += Q * Q * NE) {
    sB[i] = Bg[i];
    sG[i] = Gg[i];
  }
  const int e = blockIdx.x * NE + tz;
  const bool valid = e < ne;
  double* s = sm + tz * SE;
  double* sX = s;
  double* sBX = s + ND;
  double* sGX = sBX + D1 * D1 * Q;
  double* sR = sGX + D1 * D1 * Q;
  if (valid && tx < D1 && ty < D1)
    for (int z = 0; z < D1; ++z) {
      const int k = (z * D1 + ty) * D1 + tx;
      sX[k] = u[e2l[(size_t)e * ND + k]];
    }
  __syncthreads();
  if (ty < D1)
    for (int z = 0; z < D1; ++z) {
      double a = 0, b = 0;
      for (int d = 0; d < D1; ++d) {
        const double xv = sX[(z * D1 + ty) * D1 + d];
        a += sB[tx * D1 + d] * xv;
        b += sG[tx * D1 + d] * xv;
      }
      sBX[(z * D1 + ty) * Q + tx] = a;
      sGX[(z * D1 + ty) * Q + tx] = b;
    }
  __syncthreads();
  double rbb[D1], rgb[D1], rbg[D1];
  for (int z = 0; z < D1; ++z) {
    double bb = 0, gb = 0, bg = 0;
    for (int d = 0; d < D1; ++d) {
      const double a = sBX[(z * D1 + d) * Q + tx], b = sGX[(z * D1 + d) * Q + tx];
      bb += sB[ty * D1 + d] * a;
      gb += sB[ty * D1 + d] * b;
      bg += sG[ty * D1 + d] * a;
    }
    rbb[z] = bb;
    rgb[z] = gb;
    rbg[z] = bg;
  }
  double acc = 0.0;
  if (valid) {
    const double* De = Dq + ((size_t)e * NQ + ty * Q + tx) * 6;
    for (int qz = 0; qz < Q; ++qz) {
      double g0 = 0, g1 = 0, g2 = 0;
      for (int z = 0; z < D1; ++z) {
        g0 += sB[qz * D1 + z] * rgb[z];
        g1 += sB[qz * D1 + z] * rbg[z];
        g2 += sG[qz * D1 + z] * rbb[z];
      }
      const double* d = De + (size_t)qz * Q * Q * 6;
      const double d00 = d[0], d01 = d[1], d02 = d[2], d11 = d[3], d12 = d[4], d22 = d[5];
      acc += g0 * (d00 * g0 + d01 * g1 + d02 * g2) + g1 * (d01 * g0 + d11 * g1 + d12 * g2) +
             g2 * (d02 * g0 + d12 * g1 + d22 * g2);
    }
  }
  sR[ty * Q + tx] = acc;
  __syncthreads();
  if (valid && tx == 0 && ty == 0) {
    double sum = 0.0;
    for (int i = 0; i < Q * Q; ++i) sum += sR[i];
    g[e] = -sum / coef[e];
  }
}

__global__ void k_set_ess(int64_t ndof, const uint8_t* __restrict__ mask, double* __restrict__ v, double val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof; i += (int64_t)gridDim.x * blockDim.x)
    if (mask[i]) v[i] = val;
}

__global__ void k_keep_ess(int64_t ndof, const uint8_t* __restrict__ mask, const double* __restrict__ g,
                           double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mask[i] ? g[i] : 0.0;
}

__global__ void k_lift(int64_t ndof, const uint8_t* __restrict__ mask, const double* __restrict__ b,
                       const double* __restrict__ ag, const double* __restrict__ g, double* __restrict__ bc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof; i += (int64_t)gridDim.x * blockDim.x)
    bc[i] = mask[i] ? g[i] : b[i] - ag[i];
}

template <typename K>
fem_status set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    FEM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return FEM_OK;
}

// kind FEM_DIFFUSION reads D as [ne][nq][6], FEM_MASS as [ne][nq].
template <int P, int Q>
fem_status launch_diag(const fem_form* f, const double* D, int kind, double* ye, cudaStream_t s) {
  constexpr int D1 = P + 1, NE = ne_per_block_aux(P);
  const int ne = (int)f->space->ne;
  const size_t bytes = sizeof(double) * NE * (D1 * Q * Q + 3 * D1 * D1 * Q);
  auto k = k_diag<D1, Q, NE>;
  FEM_TRY(set_smem(k, bytes));
  k<<<(ne + NE - 1) / NE, dim3(Q, Q, NE), bytes, s>>>(ne, kind, D, f->d_B, f->d_G, ye);
  FEM_LAUNCHED();
  return FEM_OK;
}

template <int P, int Q>
fem_status launch_rhs(const fem_form* f, const double* fq, double* ye, cudaStream_t s) {
  constexpr int D1 = P + 1, NE = ne_per_block_aux(P);
  const int ne = (int)f->space->ne;
  const size_t bytes = sizeof(double) * NE * (D1 * Q * Q + D1 * D1 * Q + 24);
  auto k = k_rhs<D1, Q, NE>;
  FEM_TRY(set_smem(k, bytes));
  const fem_mesh* m = f->space->mesh;
  NodalGeo ng{nullptr, nullptr, nullptr, 0, nullptr};
  if (m->geo_k > 0) {
    FEM_TRY(fem_form_geo_tables(f));
    ng = NodalGeo{m->d_gnodes, f->d_gB, f->d_gG, m->geo_k + 1, nullptr};
  }
  k<<<(ne + NE - 1) / NE, dim3(Q, Q, NE), bytes, s>>>(ne, m->d_coords, m->d_hex, f->d_qpts, f->d_qwts, f->d_B, fq,
                                                      ye, ng);
  FEM_LAUNCHED();
  return FEM_OK;
}

template <int P, int Q>
fem_status launch_grad(const fem_form* f, const double* u, double* g, cudaStream_t s) {
  constexpr int D1 = P + 1, NE = ne_per_block_aux(P);
  const int ne = (int)f->space->ne;
  const size_t bytes = sizeof(double) * NE * (D1 * D1 * D1 + 2 * D1 * D1 * Q + Q * Q);
  auto k = k_grad<D1, Q, NE>;
  FEM_TRY(set_smem(k, bytes));
  k<<<(ne + NE - 1) / NE, dim3(Q, Q, NE), bytes, s>>>(ne, f->space->d_e2l, f->d_D, f->d_coef, f->d_B, f->d_G, u, g);
  FEM_LAUNCHED();
  return FEM_OK;
}

}  // namespace

static fem_status diag_pq(const fem_form* f, const double* D, int kind, double* ye, cudaStream_t s) {
  const int p = f->space->p, q = f->q1d;
#define X(P, Q) \
  if (p == P && q == Q) return launch_diag<P, Q>(f, D, kind, ye, s);
  FEM_FOR_EACH_PQ(X)
#undef X
  return fem_fail(FEM_EUNSUPPORTED, "diag: (p=%d, q1d=%d) not compiled", p, q);
}

fem_status fem_launch_diag_element(const fem_form* f, double* ye, cudaStream_t s) {
  if (f->space->mesh->dim == 2) return fem_launch_diag_element_2d(f, ye, s);
  if (f->kind != FEM_ELASTICITY) return diag_pq(f, f->d_D, f->kind, ye, s);
  // elasticity: the (c, c) block's diagonal is the diffusion diagonal with
  // the per-point matrix D^c; one temporary [ne][nq][6] reused for c = 0..2
  double* Dc = nullptr;
  FEM_TRY(dev_alloc(&Dc, (size_t)f->space->ne * f->nq * 6));
  fem_status st = FEM_OK;
  const size_t nend = (size_t)f->space->ne * f->space->nd;
  for (int c = 0; c < 3 && st == FEM_OK; ++c) {
    st = fem_launch_elasticity_diag_D(f, c, Dc, s);
    if (st == FEM_OK) st = diag_pq(f, Dc, FEM_DIFFUSION, ye + c * nend, s);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && st == FEM_OK)
    st = fem_fail(FEM_ECUDA, "diag: %s", cudaGetErrorString(cudaGetLastError()));
  dev_free(Dc);
  return st;
}

fem_status fem_launch_rhs_element(const fem_form* f, const double* fq, double* ye, cudaStream_t s) {
  if (f->space->mesh->dim == 2) return fem_launch_rhs_element_2d(f, fq, ye, s);
  const int p = f->space->p, q = f->q1d;
  // vector forms: component c of fq [vdim][ne][nq] into ye [vdim][ne][nd]
  const size_t nq = (size_t)f->space->ne * f->nq, nend = (size_t)f->space->ne * f->space->nd;
  for (int c = 0; c < f->vdim; ++c) {
    bool done = false;
    fem_status st = FEM_OK;
#define X(P, Q)                                                \
  if (!done && p == P && q == Q) {                             \
    st = launch_rhs<P, Q>(f, fq + c * nq, ye + c * nend, s);   \
    done = true;                                               \
  }
    FEM_FOR_EACH_PQ(X)
#undef X
    if (!done) return fem_fail(FEM_EUNSUPPORTED, "rhs: (p=%d, q1d=%d) not compiled", p, q);
    if (st != FEM_OK) return st;
  }
  return FEM_OK;
}

fem_status fem_launch_grad(const fem_form* f, const double* u, double* g, cudaStream_t s) {
  if (f->space->mesh->dim == 2) return fem_launch_grad_2d(f, u, g, s);
  const int p = f->space->p, q = f->q1d;
#define X(P, Q) \
  if (p == P && q == Q) return launch_grad<P, Q>(f, u, g, s);
  FEM_FOR_EACH_PQ(X)
#undef X
  return fem_fail(FEM_EUNSUPPORTED, "grad: (p=%d, q1d=%d) not compiled", p, q);
}

extern "C" fem_status fem_assemble_diagonal(const fem_form* f, double* diag, int constrained, void* stream) {
  if (!f || !diag) return fem_fail(FEM_EINVAL, "fem_assemble_diagonal: NULL argument");
  if (f->kind == FEM_CONVECTION) return fem_fail(FEM_EUNSUPPORTED, "fem_assemble_diagonal: convection form");
  if (constrained && !f->d_ess_mask)
    return fem_fail(FEM_EINVAL, "fem_assemble_diagonal: constrained diagonal needs fem_form_set_essential");
  cudaStream_t s = (cudaStream_t)stream;
  FEM_TRY(fem_launch_diag_element(f, (double*)f->d_ye, s));
  FEM_TRY(fem_launch_scatter(f, FEM_F64, f->d_ye, diag, nullptr, nullptr, nullptr, 0, s));
  if (constrained) {
    const int64_t n = fem_form_len(f);
    k_set_ess<<<grid_for(n, 256), 256, 0, s>>>(n, f->d_ess_mask, diag, 1.0);
    FEM_LAUNCHED();
  }
  return FEM_OK;
}

extern "C" fem_status fem_rhs(const fem_form* f, const double* fq, double* b, void* stream) {
  if (!f || !fq || !b) return fem_fail(FEM_EINVAL, "fem_rhs: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  FEM_TRY(fem_launch_rhs_element(f, fq, (double*)f->d_ye, s));
  return fem_launch_scatter(f, FEM_F64, f->d_ye, b, nullptr, nullptr, nullptr, 0, s);
}

extern "C" fem_status fem_compliance_grad(const fem_form* f, const double* u, double* g, void* stream) {
  if (!f || !u || !g) return fem_fail(FEM_EINVAL, "fem_compliance_grad: NULL argument");
  if (f->kind != FEM_DIFFUSION) return fem_fail(FEM_EINVAL, "fem_compliance_grad: needs a diffusion form");
  return fem_launch_grad(f, u, g, (cudaStream_t)stream);
}

extern "C" fem_status fem_lift_rhs(const fem_form* fc, const double* b, const double* g, double* bc, void* stream) {
  if (!fc || !b || !g || !bc) return fem_fail(FEM_EINVAL, "fem_lift_rhs: NULL argument");
  if (!fc->d_ess_mask) return fem_fail(FEM_EINVAL, "fem_lift_rhs: needs fem_form_set_essential");
  if (bc == b || bc == g) return fem_fail(FEM_EINVAL, "fem_lift_rhs: bc must not alias b or g");
  fem_form* f = const_cast<fem_form*>(fc);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = fem_form_len(f);
  // scratch: [0,n) essential part of g, [n,2n) A applied to it
  if (f->work64_len < (size_t)2 * n) {
    dev_free(f->d_work64);
    FEM_TRY(dev_alloc(&f->d_work64, (size_t)2 * n));
    f->work64_len = (size_t)2 * n;
  }
  double* ge = f->d_work64;
  double* ag = f->d_work64 + n;
  k_keep_ess<<<grid_for(n, 256), 256, 0, s>>>(n, f->d_ess_mask, g, ge);
  FEM_LAUNCHED();
  FEM_TRY(fem_launch_apply_element(f, FEM_F64, ge, f->d_ye, s));
  FEM_TRY(fem_launch_scatter(f, FEM_F64, f->d_ye, ag, nullptr, nullptr, nullptr, 0, s));
  k_lift<<<grid_for(n, 256), 256, 0, s>>>(n, f->d_ess_mask, b, ag, g, bc);
  FEM_LAUNCHED();
  return FEM_OK;
}
