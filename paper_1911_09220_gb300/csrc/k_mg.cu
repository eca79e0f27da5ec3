// p-multigrid preconditioner and flexible CG on the partially assembled
// operator. The paper names matrix-free p-multigrid for PA operators (Sec.
// 5.2, the paragraph on matrix-free preconditioners) without an algorithm;
// the one implemented here:
//
//   levels      orders p, p/2, ..., 1 on the same mesh and coefficient, each
//               a PA form with q_l = p_l + (q - p) Gauss points;
//   essential   a coarse DOF is essential iff every fine DOF of the same mesh
//               entity (vertex, edge, face, interior of an element) is;
//   transfers   P: nodal interpolation of the coarse function at the fine GLL
//               nodes, the row of fine DOF i taken from the first element
//               slot that holds i (the inverse map's first entry); masked
//               P~ = (I - E_f) P (I - E_c), restriction P~^T. Both run as
//               sum-factorized element contractions with the 1D matrix
//               I[i][j] = l^c_j(x^f_i): prolongation gathers the coarse
//               values of each element, contracts, and every fine DOF picks
//               its first slot; restriction spreads each fine residual to its
//               first slot only, contracts with I^T, and the coarse inverse
//               map sums;
//   smoother    K Chebyshev steps with Jacobi preconditioning (Saad, Iterative
//               Methods for Sparse Linear Systems, Alg. 12.1) on
//               [cheb_lo, 1] * cheb_hi * lambda, lambda = the D-Rayleigh
//               quotient after power iterations on D^-1 A_c (the operator
//               applied in double-float);
//   coarsest    a fixed number of Jacobi-PCG iterations from zero;
//   outer       flexible CG (Notay 2000; beta = z.(r - r_old) / z_old.r_old)
//               in FP64, the V-cycle in FP64 or FP32.
//   vector      elasticity forms: every level is an elasticity form with the
//               same Lame coefficients; the essential rule and the transfers
//               act on each component separately (P = blockdiag(P, P, P) on
//               component-major vectors); smoother, coarsest CG and outer
//               iteration run on the whole vector.
//
// Every kernel takes the outer iteration's `done` word and returns at once
// when it is set, so whole outer iterations (V-cycle included) are captured
// in a CUDA graph and replayed between host polls, as in the PCG solver.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

#include "fem_internal.h"
#include "k_common.cuh"

namespace {

constexpr int kRed = 256;

struct MgScalars {
  double rz, alpha, beta, rr, tol2;
  int it, done, status, maxit;
};
enum { MS_RUN = 0, MS_CONV = 1, MS_NOCONV = 2, MS_BREAK = 3 };

__device__ double sum_part(const double* part, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  return block_sum(v, red);
}

#define GRID_LOOP(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------- vector kernels
template <typename TO, typename TI>
__global__ void k_mg_in(int64_t n, const TI* __restrict__ a, const uint8_t* __restrict__ ess, TO* __restrict__ b,
                        const int* __restrict__ skip) {
  if (skip && *skip) return;
  GRID_LOOP(i, n) b[i] = ess[i] ? TO(0) : (TO)a[i];
}

template <typename TO, typename TI>
__global__ void k_mg_out(int64_t n, const TI* __restrict__ a, TO* __restrict__ b, const int* __restrict__ skip) {
  if (skip && *skip) return;
  GRID_LOOP(i, n) b[i] = (TO)a[i];
}

// pre-smoothing start: res = r, d = r / (theta D), z = d
template <typename T>
__global__ void k_cheb_pre(int64_t n, const T* __restrict__ r, const T* __restrict__ D, T inv_theta,
                           T* __restrict__ res, T* __restrict__ d, T* __restrict__ z, const int* __restrict__ skip) {
  if (*skip) return;
  GRID_LOOP(i, n) {
    const T ri = r[i];
    const T di = ri / D[i] * inv_theta;
    res[i] = ri;
    d[i] = di;
    z[i] = di;
  }
}

// post-smoothing start: res = r - A z (q = A z), d = res / (theta D), z += d
template <typename T>
__global__ void k_cheb_post(int64_t n, const T* __restrict__ r, const T* __restrict__ q, const T* __restrict__ D,
                            T inv_theta, T* __restrict__ res, T* __restrict__ d, T* __restrict__ z,
                            const int* __restrict__ skip) {
  if (*skip) return;
  GRID_LOOP(i, n) {
    const T ri = r[i] - q[i];
    const T di = ri / D[i] * inv_theta;
    res[i] = ri;
    d[i] = di;
    z[i] += di;
  }
}

// step: res -= A d (q), d = c1 d + c2 res / D, z += d
template <typename T>
__global__ void k_cheb_step(int64_t n, const T* __restrict__ q, const T* __restrict__ D, T c1, T c2,
                            T* __restrict__ res, T* __restrict__ d, T* __restrict__ z, const int* __restrict__ skip) {
  if (*skip) return;
  GRID_LOOP(i, n) {
    const T ri = res[i] - q[i];
    const T di = c1 * d[i] + c2 * (ri / D[i]);
    res[i] = ri;
    d[i] = di;
    z[i] += di;
  }
}

template <typename T>
__global__ void k_mg_sub(int64_t n, const T* __restrict__ q, T* __restrict__ res, const int* __restrict__ skip) {
  if (*skip) return;
  GRID_LOOP(i, n) res[i] -= q[i];
}

// Restriction, first half: every fine residual goes to its first slot only
// (ye[s] = r_i if s is DOF i's first slot and i is free, else 0).
template <typename T>
__global__ void k_mg_spread(int64_t nslots, const int32_t* __restrict__ e2l, const int32_t* __restrict__ off,
                            const int32_t* __restrict__ idx, const uint8_t* __restrict__ ess, const T* __restrict__ r,
                            T* __restrict__ ye, const int* __restrict__ skip) {
  if (*skip) return;
  GRID_LOOP(s, nslots) {
    const int32_t i = e2l[s];
    ye[s] = (idx[off[i]] == (int32_t)s && !ess[i]) ? r[i] : T(0);
  }
}

// FP64 <-> FP32 copies of the outer iteration's p and q (skip-aware, so
// that captured iterations after convergence do nothing).
__global__ void k_p_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b,
                           const int* __restrict__ skip) {
  if (*skip) return;
  GRID_LOOP(i, n) b[i] = (float)a[i];
}
__global__ void k_q_to_f64(int64_t n, const float* __restrict__ a, double* __restrict__ b,
                           const int* __restrict__ skip) {
  if (*skip) return;
  GRID_LOOP(i, n) b[i] = (double)a[i];
}

// dst_i = src_i on essential DOFs.
__global__ void k_copy_ess(int64_t n, const uint8_t* __restrict__ ess, const double* __restrict__ src,
                           double* __restrict__ dst) {
  GRID_LOOP(i, n) {
    if (ess[i]) dst[i] = src[i];
  }
}

// Prolongation, second half: z_i += (free i) ? ye[first slot of i] : 0
template <typename T>
__global__ void k_mg_pick(int64_t n, const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                          const uint8_t* __restrict__ ess, const T* __restrict__ ye, T* __restrict__ z,
                          const int* __restrict__ skip) {
  if (*skip) return;
  GRID_LOOP(i, n) {
    if (!ess[i]) z[i] += ye[idx[off[i]]];
  }
}

// Element-wise tensor contraction out_e = (M x M x M) in_e, M [DB][DA]
// (row-major, FP64 in global memory, cast to T in shared memory). GATHER:
// in_e[a] = (ess[map[a]] ? 0 : in[map[a]]) from an L-vector, else in is an
// E-vector [ne][DA^3]. Stages contract x, then y, then z; NE elements per
// block of 128 threads.
template <int DA, int DB>
struct InterpPlan {
  static constexpr int S0 = DA * DA * DA, S1 = DA * DA * DB, S2 = DA * DB * DB, S3 = DB * DB * DB;
  static constexpr int PER = S0 + S1 + S2;
  static constexpr int NE = PER * 8 > 16384 ? 1 : (16384 / (PER * 8) > 16 ? 16 : 16384 / (PER * 8));
};

template <typename T, int DA, int DB, bool GATHER>
__global__ void __launch_bounds__(128)
k_mg_interp(int ne, const int32_t* __restrict__ map, const uint8_t* __restrict__ ess, const T* __restrict__ in,
            const double* __restrict__ M, T* __restrict__ out, const int* __restrict__ skip) {
  using P = InterpPlan<DA, DB>;
  constexpr int NE = P::NE;
  if (*skip) return;
  __shared__ T sM[DB * DA];
  __shared__ T s0[NE * P::S0];
  __shared__ T s1[NE * P::S1];
  __shared__ T s2[NE * P::S2];
  const int e0 = blockIdx.x * NE;
  for (int k = threadIdx.x; k < DB * DA; k += blockDim.x) sM[k] = (T)M[k];
  for (int k = threadIdx.x; k < NE * P::S0; k += blockDim.x) {
    const int el = k / P::S0, a = k % P::S0;
    const int64_t e = e0 + el;
    T v = T(0);
    if (e < ne) {
      if (GATHER) {
        const int32_t c = map[e * P::S0 + a];
        v = ess[c] ? T(0) : in[c];
      } else {
        v = in[e * P::S0 + a];
      }
    }
    s0[k] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NE * P::S1; k += blockDim.x) {  // [a3][a2][b1]
    const int el = k / P::S1, r = k % P::S1, b1 = r % DB, a23 = r / DB;
    const T* src = s0 + el * P::S0 + a23 * DA;
    T acc = T(0);
#pragma unroll
    for (int a1 = 0; a1 < DA; ++a1) acc += sM[b1 * DA + a1] * src[a1];
    s1[k] = acc;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NE * P::S2; k += blockDim.x) {  // [a3][b2][b1]
    const int el = k / P::S2, r = k % P::S2, b1 = r % DB, b2 = (r / DB) % DB, a3 = r / (DB * DB);
    const T* src = s1 + el * P::S1 + a3 * DA * DB + b1;
    T acc = T(0);
#pragma unroll
    for (int a2 = 0; a2 < DA; ++a2) acc += sM[b2 * DA + a2] * src[a2 * DB];
    s2[k] = acc;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NE * P::S3; k += blockDim.x) {  // [b3][b2][b1]
    const int el = k / P::S3, r = k % P::S3, b12 = r % (DB * DB), b3 = r / (DB * DB);
    const int64_t e = e0 + el;
    if (e >= ne) continue;
    const T* src = s2 + el * P::S2 + b12;
    T acc = T(0);
#pragma unroll
    for (int a3 = 0; a3 < DA; ++a3) acc += sM[b3 * DA + a3] * src[a3 * DB * DB];
    out[e * P::S3 + r] = acc;
  }
}

// ------------------------------------------------------ coarsest-level CG
// m Jacobi-PCG iterations from zero, four launches per iteration (element,
// scatter with p.q partials, update, p update) and no single-block kernel:
// every block sums the partials it needs itself, in the same fixed order, so
// all blocks hold the same alpha and beta. The r.z partials alternate between
// two buffers by iteration parity (the launch's iteration k is a kernel
// argument), so no buffer is written while another block may read it. `stop`
// is set by block 0 when p.q <= 0 (the iteration ends there, as in the
// oracle) and read by the later launches.
template <typename T>
__global__ void k_cc_init(int64_t n, const T* __restrict__ rin, const T* __restrict__ D, T* __restrict__ r,
                          T* __restrict__ z, T* __restrict__ p, T* __restrict__ x, double* __restrict__ part_rz,
                          int* __restrict__ stop, const int* __restrict__ skip) {
  __shared__ double red[32];
  if (*skip) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *stop = 1;
    return;
  }
  using A = typename DotAcc<T>::type;
  A rz = 0;
  GRID_LOOP(i, n) {
    const T ri = rin[i];
    const T zi = ri / D[i];
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
    x[i] = T(0);
    rz += (A)ri * (A)zi;
  }
  const double s = block_sum((double)rz, red);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = s;
    if (blockIdx.x == 0) *stop = 0;
  }
}

// x += a p, r -= a q, z = r / D, partials of the new r.z into part_new;
// a = rz / pq with rz = sum(part_rz), pq = sum(part_pq).
template <typename T>
__global__ void k_cc_update(int64_t n, int nb, const double* __restrict__ part_pq, const double* __restrict__ part_rz,
                            double* __restrict__ part_new, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                            const T* __restrict__ p, const T* __restrict__ q, const T* __restrict__ D,
                            int* __restrict__ stop) {
  __shared__ double red[32];
  __shared__ double sh[2];
  if (*stop) return;
  const double pq = sum_part(part_pq, nb, red);
  if (threadIdx.x == 0) sh[0] = pq;
  const double rz = sum_part(part_rz, nb, red);
  if (threadIdx.x == 0) sh[1] = rz;
  __syncthreads();
  if (!(sh[0] > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *stop = 1;
    return;
  }
  const T a = (T)(sh[1] / sh[0]);
  using A = typename DotAcc<T>::type;
  A acc = 0;
  GRID_LOOP(i, n) {
    x[i] += a * p[i];
    const T ri = r[i] - a * q[i];
    r[i] = ri;
    const T zi = ri / D[i];
    z[i] = zi;
    acc += (A)ri * (A)zi;
  }
  const double s = block_sum((double)acc, red);
  if (threadIdx.x == 0) part_new[blockIdx.x] = s;
}

// p = z + (rz_new / rz_old) p
template <typename T>
__global__ void k_cc_p(int64_t n, int nb, const double* __restrict__ part_old, const double* __restrict__ part_new,
                       const T* __restrict__ z, T* __restrict__ p, const int* __restrict__ stop) {
  __shared__ double red[32];
  __shared__ double sh[2];
  if (*stop) return;
  const double ro = sum_part(part_old, nb, red);
  if (threadIdx.x == 0) sh[0] = ro;
  const double rn = sum_part(part_new, nb, red);
  if (threadIdx.x == 0) sh[1] = rn;
  __syncthreads();
  const T b = (T)(sh[1] / sh[0]);
  GRID_LOOP(i, n) p[i] = z[i] + b * p[i];
}

// ------------------------------------------------------------- outer FCG
__global__ void k_fg_init(MgScalars* sc, const double* __restrict__ part, int nb, double rtol2_bb, int maxit) {
  // part: [rz | rr] partials
  __shared__ double red[32];
  const double rz = sum_part(part, nb, red);
  const double rr = sum_part(part + nb, nb, red);
  if (threadIdx.x == 0) {
    sc->rz = rz;
    sc->rr = rr;
    sc->tol2 = rtol2_bb;
    sc->it = 0;
    sc->maxit = maxit;
    sc->status = MS_RUN;
    sc->done = 0;
    if (!isfinite(rz) || !isfinite(rr)) {
      sc->done = 1;
      sc->status = MS_BREAK;
    } else if (rr <= sc->tol2) {
      sc->done = 1;
      sc->status = MS_CONV;
    } else if (!(rz > 0.0)) {
      sc->done = 1;
      sc->status = MS_BREAK;
    }
  }
}

__global__ void k_fg_alpha(MgScalars* sc, const double* __restrict__ part, int nb) {
  __shared__ double red[32];
  if (sc->done) return;
  const double pq = sum_part(part, nb, red);
  if (threadIdx.x == 0) {
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc->done = 1;
      sc->status = MS_BREAK;
    } else {
      sc->alpha = sc->rz / pq;
    }
  }
}

// x += a p; r_old = r; r -= a q; partials of r.r
__global__ void k_fg_update(int64_t n, const MgScalars* __restrict__ sc, double* __restrict__ x,
                            double* __restrict__ r, double* __restrict__ rold, const double* __restrict__ p,
                            const double* __restrict__ q, double* __restrict__ part) {
  __shared__ double red[32];
  if (sc->done) return;
  const double a = sc->alpha;
  double rr = 0;
  GRID_LOOP(i, n) {
    x[i] += a * p[i];
    const double ro = r[i];
    const double ri = ro - a * q[i];
    rold[i] = ro;
    r[i] = ri;
    rr += ri * ri;
  }
  const double s = block_sum(rr, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_fg_check(MgScalars* sc, const double* __restrict__ part, int nb) {
  __shared__ double red[32];
  if (sc->done) return;
  const double rr = sum_part(part, nb, red);
  if (threadIdx.x == 0) {
    sc->it += 1;
    sc->rr = rr;
    if (!isfinite(rr)) {
      sc->done = 1;
      sc->status = MS_BREAK;
    } else if (rr <= sc->tol2) {
      sc->done = 1;
      sc->status = MS_CONV;
    } else if (sc->it >= sc->maxit) {
      sc->done = 1;
      sc->status = MS_NOCONV;
    }
  }
}

// partials of z.r and z.r_old
__global__ void k_fg_dots(int64_t n, const double* __restrict__ z, const double* __restrict__ r,
                          const double* __restrict__ rold, double* __restrict__ part, const int* __restrict__ skip) {
  __shared__ double red[32];
  if (*skip) return;
  double zr = 0, zo = 0;
  GRID_LOOP(i, n) {
    const double zi = z[i];
    zr += zi * r[i];
    zo += zi * rold[i];
  }
  double s = block_sum(zr, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  s = block_sum(zo, red);
  if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = s;
}

__global__ void k_fg_beta(MgScalars* sc, const double* __restrict__ part, int nb) {
  __shared__ double red[32];
  if (sc->done) return;
  const double zr = sum_part(part, nb, red);
  const double zo = sum_part(part + nb, nb, red);
  if (threadIdx.x == 0) {
    if (!isfinite(zr) || !(zr > 0.0)) {
      sc->done = 1;
      sc->status = MS_BREAK;
    } else {
      sc->beta = (zr - zo) / sc->rz;
      sc->rz = zr;
    }
  }
}

__global__ void k_fg_p(int64_t n, const MgScalars* __restrict__ sc, const double* __restrict__ z,
                       double* __restrict__ p) {
  if (sc->done) return;
  const double b = sc->beta;
  GRID_LOOP(i, n) p[i] = z[i] + b * p[i];
}

// partials of a.b and a.a (setup: power iteration, initial r.z and r.r)
__global__ void k_dot2(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                       double* __restrict__ part) {
  __shared__ double red[32];
  double ab = 0, aa = 0;
  GRID_LOOP(i, n) {
    ab += a[i] * b[i];
    aa += a[i] * a[i];
  }
  double s = block_sum(ab, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  s = block_sum(aa, red);
  if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = s;
}

// partials of v.w, v.(D v), u.u with u = w / D (power iteration step)
__global__ void k_pow_dots(int64_t n, const double* __restrict__ v, const double* __restrict__ w,
                           const double* __restrict__ D, double* __restrict__ u, double* __restrict__ part) {
  __shared__ double red[32];
  double vw = 0, vdv = 0, uu = 0;
  GRID_LOOP(i, n) {
    const double vi = v[i];
    vw += vi * w[i];
    vdv += vi * (D[i] * vi);
    const double ui = w[i] / D[i];
    u[i] = ui;
    uu += ui * ui;
  }
  double s = block_sum(vw, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  s = block_sum(vdv, red);
  if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = s;
  s = block_sum(uu, red);
  if (threadIdx.x == 0) part[2 * gridDim.x + blockIdx.x] = s;
}

__global__ void k_sum3(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double red[32];
  for (int j = 0; j < 3; ++j) {
    const double s = sum_part(part + j * nb, nb, red);
    if (threadIdx.x == 0) out[j] = s;
  }
}

// v_i = frac(i * 2654435761 / 2^32) - 1/2 on free DOFs, 0 on essential ones
__global__ void k_hash_vec(int64_t n, const uint8_t* __restrict__ ess, double* __restrict__ v) {
  GRID_LOOP(i, n) {
    const uint64_t h = ((uint64_t)i * 2654435761ull) & 0xFFFFFFFFull;
    v[i] = ess[i] ? 0.0 : (double)h / 4294967296.0 - 0.5;
  }
}

// b = s a; may run in place (b == a), so the pointers are not restrict.
__global__ void k_scale(int64_t n, const double* a, double s, double* b) {
  GRID_LOOP(i, n) b[i] = a[i] * s;
}

__global__ void k_to_f32v(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  GRID_LOOP(i, n) b[i] = (float)a[i];
}

__global__ void k_resid(int64_t n, const double* __restrict__ b, const double* __restrict__ y,
                        double* __restrict__ r, double* __restrict__ part) {
  __shared__ double red[32];
  double rr = 0;
  GRID_LOOP(i, n) {
    const double ri = b[i] - y[i];
    r[i] = ri;
    rr += ri * ri;
  }
  const double s = block_sum(rr, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum1(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double red[32];
  const double s = sum_part(part, nb, red);
  if (threadIdx.x == 0) *out = s;
}

// ------------------------------------------ assembled order-1 coarsest level
// Element matrices of an order-1 form (D1 = 2, local node a = ax + 2 ay + 4
// az): Ke[e][a][b] = sum_q grad phi_a(q) . D_q grad phi_b(q) (diffusion,
// D point-major [q][6]) or sum_q D_q phi_a(q) phi_b(q) (mass), with the
// form's 1D tables B, G [Q][2] at its Q Gauss points.
__global__ void k_p1_element_matrices(int64_t ne, int Q, int kind, const double* __restrict__ D,
                                      const double* __restrict__ B, const double* __restrict__ G,
                                      double* __restrict__ Ke) {
  const int nq = Q * Q * Q;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ne * 64;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / 64;
    const int a = (int)((t / 8) % 8), b = (int)(t % 8);
    const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2, bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
    double v = 0.0;
    for (int qz = 0; qz < Q; ++qz)
      for (int qy = 0; qy < Q; ++qy)
        for (int qx = 0; qx < Q; ++qx) {
          const int q = qx + Q * (qy + Q * qz);
          const double Bax = B[qx * 2 + ax], Bay = B[qy * 2 + ay], Baz = B[qz * 2 + az];
          const double Bbx = B[qx * 2 + bx], Bby = B[qy * 2 + by], Bbz = B[qz * 2 + bz];
          if (kind == FEM_DIFFUSION) {
            const double ga0 = G[qx * 2 + ax] * Bay * Baz, ga1 = Bax * G[qy * 2 + ay] * Baz,
                         ga2 = Bax * Bay * G[qz * 2 + az];
            const double gb0 = G[qx * 2 + bx] * Bby * Bbz, gb1 = Bbx * G[qy * 2 + by] * Bbz,
                         gb2 = Bbx * Bby * G[qz * 2 + bz];
            const double* d = D + (e * nq + q) * 6;
            v += ga0 * (d[0] * gb0 + d[1] * gb1 + d[2] * gb2) + ga1 * (d[1] * gb0 + d[3] * gb1 + d[4] * gb2) +
                 ga2 * (d[2] * gb0 + d[4] * gb1 + d[5] * gb2);
          } else {
            v += D[e * nq + q] * (Bax * Bay * Baz) * (Bbx * Bby * Bbz);
          }
        }
    Ke[t] = v;
  }
}

// CSR values of the constrained operator A_c = (I - E) A (I - E) + E: entry j
// (row i, column c) sums its element contributions Ke[cidx[k]], k in
// [coff[j], coff[j+1]), in ascending element order; rows and columns of
// essential DOFs are zero except the unit diagonal.
__global__ void k_csr_assemble(int64_t nnz, const int32_t* __restrict__ row_of, const int32_t* __restrict__ cols,
                               const int32_t* __restrict__ coff, const int32_t* __restrict__ cidx,
                               const double* __restrict__ Ke, const uint8_t* __restrict__ ess,
                               double* __restrict__ v64, float* __restrict__ v32) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = row_of[j], c = cols[j];
    double v = 0.0;
    if (ess[i] || ess[c]) {
      v = (i == c) ? 1.0 : 0.0;
    } else {
      for (int32_t k = coff[j]; k < coff[j + 1]; ++k) v += Ke[cidx[k]];
    }
    v64[j] = v;
    v32[j] = (float)v;
  }
}

// y = A x on the assembled level (8 lanes per row, the row's sum reduced by
// a fixed butterfly) and per-block partials of x . y; skipped when *skip.
template <typename T>
__global__ void __launch_bounds__(256)
k_csr_apply(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cols, const T* __restrict__ vals,
            const T* __restrict__ x, T* __restrict__ y, double* __restrict__ part, const int* __restrict__ skip) {
  __shared__ double red[32];
  if (skip && *skip) return;
  using A = typename DotAcc<T>::type;
  A acc = 0;
  const int lane8 = threadIdx.x & 7;
  const unsigned mask = 0xffu << (threadIdx.x & 24);
  const int64_t g0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
  const int64_t gs = ((int64_t)gridDim.x * blockDim.x) >> 3;
  for (int64_t i = g0; i < n; i += gs) {
    T v = 0;
    for (int32_t k = rowptr[i] + lane8; k < rowptr[i + 1]; k += 8) v += vals[k] * x[cols[k]];
    v += __shfl_xor_sync(mask, v, 4, 8);
    v += __shfl_xor_sync(mask, v, 2, 8);
    v += __shfl_xor_sync(mask, v, 1, 8);
    if (lane8 == 0) {
      y[i] = v;
      if (part) acc += (A)x[i] * (A)v;
    }
  }
  if (part) {
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

}  // namespace

// ------------------------------------------------------------------ handle
struct MgLevel {
  const fem_form* f = nullptr;  // the level's form (level 0: the caller's)
  fem_space* sp_own = nullptr;  // owned space and form of the coarse levels
  fem_form* f_own = nullptr;
  int p = 0, D1 = 0, nd = 0;
  int vdim = 1;                 // vector components (3 for elasticity)
  int64_t n = 0;                // vector length vdim * ndof
  double lam = 0.0, inv_theta = 0.0;
  std::vector<double> c1, c2;   // Chebyshev step coefficients
  double* diag64 = nullptr;
  float* diag32 = nullptr;
  void* vec = nullptr;          // r, z, res, d, q (T each)
  double* I = nullptr;          // to the next coarser level: I [D1][D1c], I^T [D1c][D1]
  double* It = nullptr;
  // assembled constrained operator (the coarsest level when it has order 1)
  int64_t nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* cols = nullptr;
  double* vals64 = nullptr;
  float* vals32 = nullptr;
};

struct fem_mg {
  const fem_form* fine = nullptr;
  fem_mg_opts o{};
  std::vector<MgLevel> lv;
  int nb = 0;                   // vector-kernel blocks (fine level)
  void* zero = nullptr;         // zeros (T) of the largest coarse level
  void* cc_vec = nullptr;       // coarsest CG: r, z, p, q (T)
  double* part = nullptr;       // 3 * nb partials
  int* d_stop = nullptr;        // coarsest CG: stop word
  MgScalars* sc = nullptr;      // outer FCG scalars
  double* w64 = nullptr;        // FCG: x, r, rold, z, p, q, t
  float* w32 = nullptr;         // FCG with the FP32 outer operator: p, q in FP32 (lazy)
  int* h = nullptr;             // pinned host words
  int never = 0;                // device word that stays 0 (standalone V-cycle)
  int* d_never = nullptr;
};

namespace {

template <typename T>
T* lvec(const MgLevel& L, int k) {
  return reinterpret_cast<T*>(L.vec) + (size_t)k * L.n;
}

// y = A_c x on level L (x zero on essential DOFs), type T.
template <typename T>
fem_status level_apply(const MgLevel& L, const T* x, T* y, const int* skip, cudaStream_t s, double* pdot = nullptr,
                       int nb = 0) {
  const int dt = std::is_same<T, float>::value ? FEM_F32 : FEM_F64;
  FEM_TRY(fem_launch_apply_element(L.f, dt, x, L.f->d_ye, s, skip, true));
  return fem_launch_scatter(L.f, dt, L.f->d_ye, y, L.f->d_ess_mask, x, pdot, nb, s, skip, true);
}

int vblocks(int64_t n) { return grid_for(n, 256); }

// y = A_c x in double-float element arithmetic on FP64 vectors (x zero on
// essential DOFs): the lambda estimate needs no more than its ~1e-13
// accuracy, and it runs on the FP32 pipe at about 4x the FP64 apply's rate.
fem_status level_apply_df(const MgLevel& L, const double* x, double* y, const int* skip, cudaStream_t s) {
  FEM_TRY(fem_launch_apply_element(L.f, FEM_DF64, x, L.f->d_ye, s, skip, true));
  return fem_launch_scatter(L.f, FEM_F64, L.f->d_ye, y, L.f->d_ess_mask, x, nullptr, 0, s, skip, true);
}

// Dispatch of the interpolation kernel over the compiled (D1f, D1c) pairs.
template <typename T>
fem_status launch_interp(int D1f, int D1c, bool prolong, int ne, const int32_t* map, const uint8_t* ess, const T* in,
                         const double* M, T* out, const int* skip, cudaStream_t s) {
#define PAIR(F, C)                                                                                      \
  if (D1f == F && D1c == C) {                                                                           \
    if (prolong) {                                                                                      \
      constexpr int NE = InterpPlan<C, F>::NE;                                                          \
      k_mg_interp<T, C, F, true><<<(ne + NE - 1) / NE, 128, 0, s>>>(ne, map, ess, in, M, out, skip);    \
    } else {                                                                                            \
      constexpr int NE = InterpPlan<F, C>::NE;                                                          \
      k_mg_interp<T, F, C, false><<<(ne + NE - 1) / NE, 128, 0, s>>>(ne, map, ess, in, M, out, skip);   \
    }                                                                                                   \
    FEM_LAUNCHED();                                                                                     \
    return FEM_OK;                                                                                      \
  }
  PAIR(3, 2) PAIR(4, 2) PAIR(5, 3) PAIR(6, 3) PAIR(7, 4) PAIR(8, 4) PAIR(9, 5)
#undef PAIR
  return fem_fail(FEM_EUNSUPPORTED, "multigrid: no transfer for orders %d -> %d", D1f - 1, D1c - 1);
}

// Blocks of the coarsest level's vector kernels: at most two per SM, so
// that every block's own sums over the partials stay short.
int cc_blocks(int64_t n) { return std::min(grid_for(n, 256), 2 * fem_sm_count()); }

template <typename T>
fem_status coarse_solve(fem_mg* m, const MgLevel& C, const int* skip, cudaStream_t s) {
  const int64_t n = C.n;
  const int nb = cc_blocks(n);
  T* cv = reinterpret_cast<T*>(m->cc_vec);
  T *r = cv, *z = cv + n, *p = cv + 2 * n, *q = cv + 3 * n;
  const T* D = std::is_same<T, float>::value ? (const T*)C.diag32 : (const T*)C.diag64;
  T* x = lvec<T>(C, 1);
  double* pq = m->part;
  double* rzp[2] = {m->part + nb, m->part + 2 * nb};
  int* stop = m->d_stop;
  k_cc_init<T><<<nb, 256, 0, s>>>(n, lvec<T>(C, 0), D, r, z, p, x, rzp[0], stop, skip);
  FEM_LAUNCHED();
  for (int k = 0; k < m->o.coarse_its; ++k) {
    if (C.nnz > 0) {
      const T* vals = std::is_same<T, float>::value ? (const T*)C.vals32 : (const T*)C.vals64;
      k_csr_apply<T><<<nb, 256, 0, s>>>(n, C.rowptr, C.cols, vals, p, q, pq, stop);
    } else {
      FEM_TRY(level_apply<T>(C, p, q, stop, s, pq, nb));
    }
    k_cc_update<T><<<nb, 256, 0, s>>>(n, nb, pq, rzp[k & 1], rzp[(k + 1) & 1], x, r, z, p, q, D, stop);
    k_cc_p<T><<<nb, 256, 0, s>>>(n, nb, rzp[k & 1], rzp[(k + 1) & 1], z, p, stop);
    FEM_LAUNCHED();
  }
  return FEM_OK;
}

// z_l = V(r_l): level vectors 0 (r) and 1 (z).
template <typename T>
fem_status vcycle(fem_mg* m, size_t l, const int* skip, cudaStream_t s) {
  const MgLevel& L = m->lv[l];
  if (l + 1 == m->lv.size()) return coarse_solve<T>(m, L, skip, s);
  const int64_t n = L.n;
  const int nb = vblocks(n);
  T *r = lvec<T>(L, 0), *z = lvec<T>(L, 1), *res = lvec<T>(L, 2), *d = lvec<T>(L, 3), *q = lvec<T>(L, 4);
  const T* D = std::is_same<T, float>::value ? (const T*)L.diag32 : (const T*)L.diag64;
  const T it = (T)L.inv_theta;
  const int K1 = (int)L.c1.size();
  // pre-smoothing from zero, then res = r - A z
  k_cheb_pre<T><<<nb, 256, 0, s>>>(n, r, D, it, res, d, z, skip);
  FEM_LAUNCHED();
  for (int k = 0; k < K1; ++k) {
    FEM_TRY(level_apply<T>(L, d, q, skip, s));
    k_cheb_step<T><<<nb, 256, 0, s>>>(n, q, D, (T)L.c1[k], (T)L.c2[k], res, d, z, skip);
    FEM_LAUNCHED();
  }
  FEM_TRY(level_apply<T>(L, d, q, skip, s));
  k_mg_sub<T><<<nb, 256, 0, s>>>(n, q, res, skip);
  FEM_LAUNCHED();
  // restriction: coarse r = P~^T res
  const MgLevel& C = m->lv[l + 1];
  const fem_space* sf = L.f->space;
  const fem_space* sc = C.f->space;
  T* yef = reinterpret_cast<T*>(L.f->d_ye);
  T* yec = reinterpret_cast<T*>(C.f->d_ye);
  // (vector forms: each component through the scalar transfer, on its
  // slices of the L-vectors, masks and E-vectors)
  const int64_t nslots = sf->ne * (int64_t)sf->nd, cslots = sc->ne * (int64_t)sc->nd;
  const int64_t nf = sf->ndof, nc = sc->ndof;
  for (int c = 0; c < L.vdim; ++c) {
    k_mg_spread<T><<<grid_for(nslots, 256), 256, 0, s>>>(nslots, sf->d_e2l, sf->d_l2e_off, sf->d_l2e_idx,
                                                         L.f->d_ess_mask + c * nf, res + c * nf, yef + c * nslots,
                                                         skip);
    FEM_LAUNCHED();
    FEM_TRY(launch_interp<T>(L.D1, C.D1, false, (int)sf->ne, nullptr, nullptr, yef + c * nslots, L.It,
                             yec + c * cslots, skip, s));
  }
  const int dt = std::is_same<T, float>::value ? FEM_F32 : FEM_F64;
  FEM_TRY(fem_launch_scatter(C.f, dt, yec, lvec<T>(C, 0), C.f->d_ess_mask, m->zero, nullptr, 0, s, skip));
  // coarse correction
  FEM_TRY(vcycle<T>(m, l + 1, skip, s));
  // prolongation: z += P~ z_c
  for (int c = 0; c < L.vdim; ++c) {
    FEM_TRY(launch_interp<T>(L.D1, C.D1, true, (int)sf->ne, sc->d_e2l, C.f->d_ess_mask + c * nc,
                             lvec<T>(C, 1) + c * nc, L.I, yef + c * nslots, skip, s));
    k_mg_pick<T><<<vblocks(nf), 256, 0, s>>>(nf, sf->d_l2e_off, sf->d_l2e_idx, L.f->d_ess_mask + c * nf,
                                             yef + c * nslots, z + c * nf, skip);
    FEM_LAUNCHED();
  }
  // post-smoothing from z
  FEM_TRY(level_apply<T>(L, z, q, skip, s));
  k_cheb_post<T><<<nb, 256, 0, s>>>(n, r, q, D, it, res, d, z, skip);
  FEM_LAUNCHED();
  for (int k = 0; k < K1; ++k) {
    FEM_TRY(level_apply<T>(L, d, q, skip, s));
    k_cheb_step<T><<<nb, 256, 0, s>>>(n, q, D, (T)L.c1[k], (T)L.c2[k], res, d, z, skip);
    FEM_LAUNCHED();
  }
  return FEM_OK;
}

// z = M^-1 r for FP64 vectors r, z of the fine level.
fem_status precond(fem_mg* m, const double* r, double* z, const int* skip, cudaStream_t s) {
  const MgLevel& L = m->lv[0];
  const int nb = vblocks(L.n);
  if (m->o.precision == FEM_F32) {
    k_mg_in<float, double><<<nb, 256, 0, s>>>(L.n, r, L.f->d_ess_mask, lvec<float>(L, 0), skip);
    FEM_LAUNCHED();
    FEM_TRY(vcycle<float>(m, 0, skip, s));
    k_mg_out<double, float><<<nb, 256, 0, s>>>(L.n, lvec<float>(L, 1), z, skip);
  } else {
    k_mg_in<double, double><<<nb, 256, 0, s>>>(L.n, r, L.f->d_ess_mask, lvec<double>(L, 0), skip);
    FEM_LAUNCHED();
    FEM_TRY(vcycle<double>(m, 0, skip, s));
    k_mg_out<double, double><<<nb, 256, 0, s>>>(L.n, lvec<double>(L, 1), z, skip);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status power_lambda_iterate(fem_mg* m, MgLevel& L, double* v, double* w, double* u, cudaStream_t s);

fem_status read_words(fem_mg* m, const void* d, size_t bytes, void* out, cudaStream_t s) {
  FEM_CUDA(cudaMemcpyAsync(m->h, d, bytes, cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  std::memcpy(out, m->h, bytes);
  return FEM_OK;
}

// lambda of D^-1 A_c on level L (double-float operator, FP64 vectors and
// dot products), power iterations as in the module header; uses the level's
// FP64 scratch w64 (4 n doubles). A double-float copy of D made only for
// this is freed again.
fem_status power_lambda(fem_mg* m, MgLevel& L, double* v, double* w, double* u, cudaStream_t s) {
  const bool had_df = L.f->d_Ddf != nullptr;
  fem_status st = power_lambda_iterate(m, L, v, w, u, s);
  if (!had_df) {
    fem_form* f = const_cast<fem_form*>(L.f);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == FEM_OK)
      st = fem_fail(FEM_ECUDA, "multigrid: lambda estimate failed");
    dev_free(f->d_Ddf);
  }
  return st;
}

fem_status power_lambda_iterate(fem_mg* m, MgLevel& L, double* v, double* w, double* u, cudaStream_t s) {
  const int64_t n = L.n;
  const int nb = vblocks(n);
  const int* never = m->d_never;
  k_hash_vec<<<nb, 256, 0, s>>>(n, L.f->d_ess_mask, v);
  k_dot2<<<nb, 256, 0, s>>>(n, v, v, m->part);
  double* sums = m->part + 3 * m->nb;
  k_sum3<<<1, kRed, 0, s>>>(m->part, nb, sums);  // (v.v, v.v, -)
  FEM_LAUNCHED();
  double hs[3];
  FEM_TRY(read_words(m, sums, sizeof hs, hs, s));
  if (!(hs[0] > 0.0)) {
    L.lam = 1.0;  // no free DOFs: any interval will do
    return FEM_OK;
  }
  k_scale<<<nb, 256, 0, s>>>(n, v, 1.0 / std::sqrt(hs[0]), v);
  FEM_LAUNCHED();
  double lam = 0.0;
  for (int it = 0; it < m->o.power_its; ++it) {
    FEM_TRY(level_apply_df(L, v, w, never, s));
    k_pow_dots<<<nb, 256, 0, s>>>(n, v, w, L.diag64, u, m->part);
    k_sum3<<<1, kRed, 0, s>>>(m->part, nb, sums);
    FEM_LAUNCHED();
    FEM_TRY(read_words(m, sums, sizeof hs, hs, s));
    if (!(hs[1] > 0.0) || !(hs[2] > 0.0) || !std::isfinite(hs[0])) break;
    lam = hs[0] / hs[1];
    k_scale<<<nb, 256, 0, s>>>(n, u, 1.0 / std::sqrt(hs[2]), v);
    FEM_LAUNCHED();
  }
  L.lam = lam > 0.0 ? lam : 1.0;
  return FEM_OK;
}

void cheb_setup(MgLevel& L, const fem_mg_opts& o) {
  const double hi = o.cheb_hi * L.lam, lo = o.cheb_lo * hi;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  L.inv_theta = 1.0 / theta;
  L.c1.clear();
  L.c2.clear();
  for (int k = 1; k < o.cheb_order; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    L.c1.push_back(rn * rho);
    L.c2.push_back(2.0 * rn / delta);
    rho = rn;
  }
}

// Assemble the order-1 coarsest level into CSR (once, at set-up). Pattern:
// row i holds the DOFs of the elements containing DOF i, ascending. Each
// element-matrix entry (e, a, b) contributes to (e2l[e][a], e2l[e][b]); the
// contributions of an entry are summed in ascending element order, so the
// values do not depend on the schedule.
// fn(i0, i1) over [0, n) in contiguous ranges on up to 16 host threads.
template <typename F>
void host_parallel(int64_t n, F fn) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), 16, n / 8192 + 1}));
  if (nt == 1) {
    fn((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t) th.emplace_back(fn, n * t / nt, n * (t + 1) / nt);
  for (auto& x : th) x.join();
}

fem_status assemble_coarse(MgLevel& C, cudaStream_t s) {
  const fem_space* sp = C.f->space;
  const int64_t ne = sp->ne, n = sp->ndof;
  const std::vector<int32_t>& e2l = sp->e2l;
  std::vector<int32_t> eoff(n + 1, 0), eslot((size_t)ne * 8);
  for (int64_t k = 0; k < ne * 8; ++k) eoff[e2l[k] + 1]++;
  for (int64_t i = 0; i < n; ++i) eoff[i + 1] += eoff[i];
  {
    std::vector<int32_t> fill(eoff.begin(), eoff.end() - 1);
    for (int64_t k = 0; k < ne * 8; ++k) eslot[fill[e2l[k]]++] = (int32_t)k;  // ascending element
  }
  for (int64_t i = 0; i < n; ++i)
    if (eoff[i + 1] - eoff[i] > 64) return FEM_EUNSUPPORTED;  // > 64 elements at a vertex: stay matrix-free
  // rows: the sorted distinct DOFs of the elements holding DOF i, counted in
  // parallel, then written at their offsets
  auto row_cols = [&](int64_t i, int32_t* out) {
    int32_t tmp[64 * 8];
    int m = 0;
    for (int32_t t = eoff[i]; t < eoff[i + 1]; ++t) {
      const int64_t e = eslot[t] / 8;
      for (int b = 0; b < 8; ++b) tmp[m++] = e2l[e * 8 + b];
    }
    std::sort(tmp, tmp + m);
    const int u = (int)(std::unique(tmp, tmp + m) - tmp);
    if (out) std::copy(tmp, tmp + u, out);
    return u;
  };
  std::vector<int32_t> rowptr(n + 1, 0);
  host_parallel(n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) rowptr[i + 1] = row_cols(i, nullptr);
  });
  for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
  const int64_t nnz = rowptr[n];
  std::vector<int32_t> cols(nnz), row_of(nnz);
  host_parallel(n, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      row_cols(i, cols.data() + rowptr[i]);
      std::fill(row_of.begin() + rowptr[i], row_of.begin() + rowptr[i + 1], (int32_t)i);
    }
  });
  // contributions: the entry of every element-matrix slot (parallel over
  // elements), then a counting sort that keeps ascending element order
  std::vector<int32_t> cpos((size_t)ne * 64);
  host_parallel(ne, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e)
      for (int a = 0; a < 8; ++a) {
        const int32_t i = e2l[e * 8 + a];
        const int32_t* rb = cols.data() + rowptr[i];
        const int32_t* re = cols.data() + rowptr[i + 1];
        for (int b = 0; b < 8; ++b)
          cpos[(size_t)e * 64 + a * 8 + b] = (int32_t)(std::lower_bound(rb, re, e2l[e * 8 + b]) - cols.data());
      }
  });
  std::vector<int32_t> coff(nnz + 1, 0);
  for (int64_t t = 0; t < ne * 64; ++t) coff[cpos[t] + 1]++;
  for (int64_t j = 0; j < nnz; ++j) coff[j + 1] += coff[j];
  std::vector<int32_t> cidx((size_t)ne * 64);
  {
    std::vector<int32_t> fill(coff.begin(), coff.end() - 1);
    for (int64_t t = 0; t < ne * 64; ++t) cidx[fill[cpos[t]]++] = (int32_t)t;
  }
  // device: element matrices, then the entries
  int32_t *d_row_of = nullptr, *d_coff = nullptr, *d_cidx = nullptr;
  double* d_Ke = nullptr;
  fem_status st = dev_alloc(&C.rowptr, rowptr.size());
  if (st == FEM_OK) st = dev_alloc(&C.cols, cols.size());
  if (st == FEM_OK) st = dev_alloc(&C.vals64, cols.size());
  if (st == FEM_OK) st = dev_alloc(&C.vals32, cols.size());
  if (st == FEM_OK) st = dev_alloc(&d_row_of, row_of.size());
  if (st == FEM_OK) st = dev_alloc(&d_coff, coff.size());
  if (st == FEM_OK) st = dev_alloc(&d_cidx, cidx.size());
  if (st == FEM_OK) st = dev_alloc(&d_Ke, (size_t)ne * 64);
  if (st == FEM_OK &&
      (cudaMemcpy(C.rowptr, rowptr.data(), sizeof(int32_t) * rowptr.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(C.cols, cols.data(), sizeof(int32_t) * cols.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_row_of, row_of.data(), sizeof(int32_t) * row_of.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_coff, coff.data(), sizeof(int32_t) * coff.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_cidx, cidx.data(), sizeof(int32_t) * cidx.size(), cudaMemcpyHostToDevice) != cudaSuccess))
    st = fem_fail(FEM_ECUDA, "fem_mg_create: upload of the coarse matrix pattern failed");
  if (st == FEM_OK) {
    k_p1_element_matrices<<<grid_for(ne * 64, 256), 256, 0, s>>>(ne, C.f->q1d, C.f->kind, C.f->d_D, C.f->d_B,
                                                                  C.f->d_G, d_Ke);
    k_csr_assemble<<<grid_for(nnz, 256), 256, 0, s>>>(nnz, d_row_of, C.cols, d_coff, d_cidx, d_Ke,
                                                       C.f->d_ess_mask, C.vals64, C.vals32);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "fem_mg_create: coarse matrix assembly failed");
  }
  dev_free(d_row_of);
  dev_free(d_coff);
  dev_free(d_cidx);
  dev_free(d_Ke);
  if (st != FEM_OK) {
    dev_free(C.rowptr);
    dev_free(C.cols);
    dev_free(C.vals64);
    dev_free(C.vals32);
    return st;
  }
  C.nnz = nnz;
  return FEM_OK;
}

template <typename T>
fem_status alloc_vecs(fem_mg* m) {
  size_t maxc = 1;
  for (size_t l = 0; l < m->lv.size(); ++l) {
    MgLevel& L = m->lv[l];
    T* v = nullptr;
    FEM_TRY(dev_alloc(&v, (size_t)5 * L.n));
    FEM_CUDA(cudaMemset(v, 0, sizeof(T) * 5 * L.n));
    L.vec = v;
    if (l > 0) maxc = std::max(maxc, (size_t)L.n);
  }
  T* z = nullptr;
  FEM_TRY(dev_alloc(&z, maxc));
  FEM_CUDA(cudaMemset(z, 0, sizeof(T) * maxc));
  m->zero = z;
  T* c = nullptr;
  FEM_TRY(dev_alloc(&c, (size_t)4 * m->lv.back().n));
  m->cc_vec = c;
  return FEM_OK;
}

}  // namespace

extern "C" void fem_mg_opts_default(fem_mg_opts* o) {
  if (!o) return;
  o->cheb_order = 2;
  o->cheb_lo = 0.25;
  o->cheb_hi = 1.1;
  o->power_its = 20;
  o->coarse_its = 30;
  o->precision = FEM_F64;
  o->coarse_assembled = 1;
}

extern "C" void fem_mg_destroy(fem_mg* m) {
  if (!m) return;
  for (MgLevel& L : m->lv) {
    dev_free(L.diag64);
    dev_free(L.diag32);
    if (L.vec) cudaFree(L.vec);
    dev_free(L.I);
    dev_free(L.It);
    dev_free(L.rowptr);
    dev_free(L.cols);
    dev_free(L.vals64);
    dev_free(L.vals32);
    if (L.f_own) fem_form_destroy(L.f_own);
    if (L.sp_own) fem_space_destroy(L.sp_own);
  }
  if (m->zero) cudaFree(m->zero);
  dev_free(m->w32);
  if (m->cc_vec) cudaFree(m->cc_vec);
  dev_free(m->part);
  dev_free(m->d_stop);
  if (m->sc) cudaFree(m->sc);
  dev_free(m->w64);
  dev_free(m->d_never);
  if (m->h) cudaFreeHost(m->h);
  delete m;
}

extern "C" fem_status fem_mg_create(const fem_form* fine, const fem_mg_opts* opts, void* stream, fem_mg** out) {
  if (!fine || !out) return fem_fail(FEM_EINVAL, "fem_mg_create: NULL argument");
  *out = nullptr;
  if (!fine->d_ess_mask) return fem_fail(FEM_EINVAL, "fem_mg_create: call fem_form_set_essential first (n may be 0)");
  if (fine->space->mesh->dim != 3) return fem_fail(FEM_EUNSUPPORTED, "fem_mg_create: hexahedral meshes only");
  if (fine->kind != FEM_MASS && fine->kind != FEM_DIFFUSION && fine->kind != FEM_ELASTICITY)
    return fem_fail(FEM_EINVAL, "fem_mg_create: needs a symmetric (mass, diffusion or elasticity) form");
  fem_mg_opts o;
  fem_mg_opts_default(&o);
  if (opts) o = *opts;
  if (o.cheb_order < 1 || o.power_its < 1 || o.coarse_its < 0 || !(o.cheb_lo > 0.0 && o.cheb_lo < 1.0) ||
      !(o.cheb_hi > 0.0) || (o.precision != FEM_F64 && o.precision != FEM_F32))
    return fem_fail(FEM_EINVAL, "fem_mg_create: bad options");
  cudaStream_t s = (cudaStream_t)stream;
  fem_mg* m = new fem_mg();
  m->fine = fine;
  m->o = o;
  fem_status st = FEM_OK;
  auto fail = [&](fem_status e) {
    fem_mg_destroy(m);
    return e;
  };
  // levels
  const fem_space* sp0 = fine->space;
  const int dq = fine->q1d - sp0->p;
  MgLevel L0;
  L0.f = fine;
  L0.p = sp0->p;
  L0.D1 = sp0->D1;
  L0.nd = sp0->nd;
  L0.vdim = fine->vdim;
  L0.n = fem_form_len(fine);
  m->lv.push_back(L0);
  const int vd = fine->vdim;
  std::vector<uint8_t> essf(L0.n);
  if (cudaMemcpy(essf.data(), fine->d_ess_mask, L0.n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(fem_fail(FEM_ECUDA, "fem_mg_create: reading the essential mask failed"));
  while (m->lv.back().p > 1) {
    const MgLevel& F = m->lv.back();
    MgLevel C;
    C.p = F.p / 2;
    if ((st = fem_space_create(sp0->mesh, C.p, &C.sp_own)) != FEM_OK) return fail(st);
    if (fine->kind == FEM_ELASTICITY)
      st = fem_form_create_elasticity(C.sp_own, C.p + dq, fine->d_coef, fine->d_mu, stream, &C.f_own);
    else
      st = fem_form_create(C.sp_own, fine->kind, C.p + dq, fine->d_coef, stream, &C.f_own);
    if (st != FEM_OK) {
      fem_space_destroy(C.sp_own);
      return fail(st);
    }
    C.f = C.f_own;
    C.D1 = C.sp_own->D1;
    C.nd = C.sp_own->nd;
    C.vdim = vd;
    C.n = vd * C.sp_own->ndof;
    // coarse essential DOFs of each component from that component's fine mask
    std::vector<int32_t> ess;
    for (int c = 0; c < vd; ++c) {
      const std::vector<int32_t> ec = fem_coarse_essential(F.f->space, essf.data() + c * F.f->space->ndof, C.sp_own);
      for (int32_t i : ec) ess.push_back(i + (int32_t)(c * C.sp_own->ndof));
    }
    int32_t* d_ess = nullptr;
    st = dev_alloc(&d_ess, ess.size());
    if (st == FEM_OK && !ess.empty() &&
        cudaMemcpy(d_ess, ess.data(), sizeof(int32_t) * ess.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "fem_mg_create: upload failed");
    if (st == FEM_OK) st = fem_form_set_essential(C.f_own, d_ess, (int64_t)ess.size(), stream);
    dev_free(d_ess);
    // 1D interpolation coarse -> fine and its transpose
    std::vector<double> nf, nc, pts, B, G;
    fem_gll_nodes(F.p, nf);
    fem_gll_nodes(C.p, nc);
    fem_lagrange_tables(nc, nf, B, G);  // B [D1f][D1c] = l^c_j(x^f_i)
    std::vector<double> Bt((size_t)C.D1 * F.D1);
    for (int i = 0; i < F.D1; ++i)
      for (int j = 0; j < C.D1; ++j) Bt[(size_t)j * F.D1 + i] = B[(size_t)i * C.D1 + j];
    MgLevel& Fm = m->lv.back();
    if (st == FEM_OK) st = dev_alloc(&Fm.I, B.size());
    if (st == FEM_OK) st = dev_alloc(&Fm.It, Bt.size());
    if (st == FEM_OK && (cudaMemcpy(Fm.I, B.data(), sizeof(double) * B.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(Fm.It, Bt.data(), sizeof(double) * Bt.size(), cudaMemcpyHostToDevice) != cudaSuccess))
      st = fem_fail(FEM_ECUDA, "fem_mg_create: upload failed");
    m->lv.push_back(C);
    if (st != FEM_OK) return fail(st);
    essf.assign(C.n, 0);
    for (int32_t i : ess) essf[i] = 1;
  }
  // the coarsest level as an assembled matrix when it has order 1 (scalar forms)
  if (o.coarse_assembled && m->lv.back().p == 1 && m->lv.back().vdim == 1 && m->lv.back().f->kind != FEM_ELASTICITY) {
    st = assemble_coarse(m->lv.back(), s);
    if (st != FEM_OK && st != FEM_EUNSUPPORTED) return fail(st);  // unsupported: the level stays matrix-free
  }
  // scratch, scalars
  const int64_t n0 = m->lv[0].n;
  m->nb = vblocks(n0);
  if ((st = dev_alloc(&m->part, (size_t)3 * m->nb + 8)) != FEM_OK) return fail(st);
  if ((st = dev_alloc(&m->d_stop, 1)) != FEM_OK) return fail(st);
  if (cudaMalloc((void**)&m->sc, sizeof(MgScalars)) != cudaSuccess)
    return fail(fem_fail(FEM_ENOMEM, "fem_mg_create: scalars"));
  FEM_CUDA(cudaMemset(m->d_stop, 0, sizeof(int)));
  FEM_CUDA(cudaMemset(m->sc, 0, sizeof(MgScalars)));
  if ((st = dev_alloc(&m->w64, (size_t)7 * n0)) != FEM_OK) return fail(st);
  if ((st = dev_alloc(&m->d_never, 1)) != FEM_OK) return fail(st);
  FEM_CUDA(cudaMemset(m->d_never, 0, sizeof(int)));
  if (cudaMallocHost((void**)&m->h, 64) != cudaSuccess) return fail(fem_fail(FEM_ENOMEM, "fem_mg_create: pinned"));
  st = o.precision == FEM_F32 ? alloc_vecs<float>(m) : alloc_vecs<double>(m);
  if (st != FEM_OK) return fail(st);
  // diagonals, FP32 copies, lambda per smoothed level
  for (size_t l = 0; l < m->lv.size(); ++l) {
    MgLevel& L = m->lv[l];
    if ((st = dev_alloc(&L.diag64, (size_t)L.n)) != FEM_OK) return fail(st);
    if ((st = fem_assemble_diagonal(L.f, L.diag64, 1, stream)) != FEM_OK) return fail(st);
    if (o.precision == FEM_F32) {
      if ((st = dev_alloc(&L.diag32, (size_t)L.n)) != FEM_OK) return fail(st);
      k_to_f32v<<<vblocks(L.n), 256, 0, s>>>(L.n, L.diag64, L.diag32);
      if (cudaGetLastError() != cudaSuccess) return fail(fem_fail(FEM_ECUDA, "fem_mg_create: launch"));
      if ((st = fem_form_ensure_f32(L.f, s)) != FEM_OK) return fail(st);
    }
    if (l + 1 < m->lv.size()) {
      double* v = m->w64;
      if ((st = power_lambda(m, L, v, v + L.n, v + 2 * L.n, s)) != FEM_OK) return fail(st);
      cheb_setup(L, o);
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(fem_fail(FEM_ECUDA, "fem_mg_create: sync"));
  *out = m;
  return FEM_OK;
}

extern "C" fem_status fem_mg_info(const fem_mg* m, int* nlevels, int* orders_host, double* lambdas_host,
                                  int64_t* ndofs_host) {
  if (!m) return fem_fail(FEM_EINVAL, "fem_mg_info: NULL handle");
  if (nlevels) *nlevels = (int)m->lv.size();
  for (size_t l = 0; l < m->lv.size(); ++l) {
    if (orders_host) orders_host[l] = m->lv[l].p;
    if (lambdas_host) lambdas_host[l] = m->lv[l].lam;
    if (ndofs_host) ndofs_host[l] = m->lv[l].n;
  }
  return FEM_OK;
}

extern "C" const fem_form* fem_mg_level_form(const fem_mg* m, int level) {
  if (!m || level < 0 || level >= (int)m->lv.size()) return nullptr;
  return m->lv[level].f;
}

extern "C" fem_status fem_mg_prolong(fem_mg* m, int level, const double* zc, double* zf, void* stream) {
  if (!m || !zc || !zf) return fem_fail(FEM_EINVAL, "fem_mg_prolong: NULL argument");
  if (level < 0 || level + 1 >= (int)m->lv.size()) return fem_fail(FEM_EINVAL, "fem_mg_prolong: bad level");
  cudaStream_t s = (cudaStream_t)stream;
  const MgLevel &L = m->lv[level], &C = m->lv[level + 1];
  const fem_space* sf = L.f->space;
  double* yef = reinterpret_cast<double*>(L.f->d_ye);
  FEM_CUDA(cudaMemsetAsync(zf, 0, sizeof(double) * L.n, s));
  const int64_t nf = sf->ndof, nc = C.f->space->ndof, nslots = sf->ne * (int64_t)sf->nd;
  for (int c = 0; c < L.vdim; ++c) {
    FEM_TRY(launch_interp<double>(L.D1, C.D1, true, (int)sf->ne, C.f->space->d_e2l, C.f->d_ess_mask + c * nc,
                                  zc + c * nc, L.I, yef + c * nslots, m->d_never, s));
    k_mg_pick<double><<<vblocks(nf), 256, 0, s>>>(nf, sf->d_l2e_off, sf->d_l2e_idx, L.f->d_ess_mask + c * nf,
                                                  yef + c * nslots, zf + c * nf, m->d_never);
    FEM_LAUNCHED();
  }
  return FEM_OK;
}

extern "C" fem_status fem_mg_restrict(fem_mg* m, int level, const double* rf, double* rc, void* stream) {
  if (!m || !rf || !rc) return fem_fail(FEM_EINVAL, "fem_mg_restrict: NULL argument");
  if (level < 0 || level + 1 >= (int)m->lv.size()) return fem_fail(FEM_EINVAL, "fem_mg_restrict: bad level");
  cudaStream_t s = (cudaStream_t)stream;
  const MgLevel &L = m->lv[level], &C = m->lv[level + 1];
  const fem_space* sf = L.f->space;
  double* yef = reinterpret_cast<double*>(L.f->d_ye);
  double* yec = reinterpret_cast<double*>(C.f->d_ye);
  const int64_t nslots = sf->ne * (int64_t)sf->nd, cslots = C.f->space->ne * (int64_t)C.f->space->nd;
  const int64_t nf = sf->ndof;
  for (int c = 0; c < L.vdim; ++c) {
    k_mg_spread<double><<<grid_for(nslots, 256), 256, 0, s>>>(nslots, sf->d_e2l, sf->d_l2e_off, sf->d_l2e_idx,
                                                              L.f->d_ess_mask + c * nf, rf + c * nf,
                                                              yef + c * nslots, m->d_never);
    FEM_LAUNCHED();
    FEM_TRY(launch_interp<double>(L.D1, C.D1, false, (int)sf->ne, nullptr, nullptr, yef + c * nslots, L.It,
                                  yec + c * cslots, m->d_never, s));
  }
  // essential rows of the coarse level: 0 (the scatter's constraint rows
  // take xin = rc itself after it was zeroed there)
  FEM_CUDA(cudaMemsetAsync(rc, 0, sizeof(double) * C.n, s));
  return fem_launch_scatter(C.f, FEM_F64, yec, rc, C.f->d_ess_mask, rc, nullptr, 0, s);
}

extern "C" fem_status fem_mg_vcycle(fem_mg* m, const double* r, double* z, void* stream) {
  if (!m || !r || !z) return fem_fail(FEM_EINVAL, "fem_mg_vcycle: NULL argument");
  return precond(m, r, z, m->d_never, (cudaStream_t)stream);
}

namespace {

// dtype: arithmetic of the outer operator apply (FEM_F64 or FEM_DF64).
fem_status fcg_iteration(fem_mg* m, int dtype, double* x, double* r, double* rold, double* z, double* p, double* q,
                         cudaStream_t s) {
  const MgLevel& L = m->lv[0];
  const int64_t n = L.n;
  const int nb = m->nb;
  const int* skip = &m->sc->done;
  if (dtype == FEM_F32) {
    // FP32 operator on the FP64 iteration: p -> FP32, FP32 apply with the
    // constrained rows and the p.q partials (accumulated in FP64), q -> FP64
    float *p32 = m->w32, *q32 = m->w32 + n;
    k_p_to_f32<<<vblocks(n), 256, 0, s>>>(n, p, p32, skip);
    FEM_LAUNCHED();
    FEM_TRY(fem_launch_apply_element(L.f, FEM_F32, p32, L.f->d_ye, s, skip, true));
    FEM_TRY(fem_launch_scatter(L.f, FEM_F32, L.f->d_ye, q32, L.f->d_ess_mask, p32, m->part, nb, s, skip, true));
    k_q_to_f64<<<vblocks(n), 256, 0, s>>>(n, q32, q, skip);
    FEM_LAUNCHED();
  } else {
    FEM_TRY(fem_launch_apply_element(L.f, dtype, p, L.f->d_ye, s, skip, true));
    FEM_TRY(fem_launch_scatter(L.f, FEM_F64, L.f->d_ye, q, L.f->d_ess_mask, p, m->part, nb, s, skip, true));
  }
  k_fg_alpha<<<1, kRed, 0, s>>>(m->sc, m->part, nb);
  k_fg_update<<<nb, 256, 0, s>>>(n, m->sc, x, r, rold, p, q, m->part);
  k_fg_check<<<1, kRed, 0, s>>>(m->sc, m->part, nb);
  FEM_LAUNCHED();
  FEM_TRY(precond(m, r, z, skip, s));
  k_fg_dots<<<nb, 256, 0, s>>>(n, z, r, rold, m->part, skip);
  k_fg_beta<<<1, kRed, 0, s>>>(m->sc, m->part, nb);
  k_fg_p<<<nb, 256, 0, s>>>(n, m->sc, z, p);
  FEM_LAUNCHED();
  return FEM_OK;
}

// r = b - A_c x (FP64), returns ||r||^2 on the host.
fem_status fine_residual(fem_mg* m, const double* b, const double* x, double* r, double* t, double* y, double* rr,
                         cudaStream_t s) {
  const MgLevel& L = m->lv[0];
  FEM_TRY(fem_launch_zero_ess(L.f, FEM_F64, x, t, s));
  FEM_TRY(fem_launch_apply_element(L.f, FEM_F64, t, L.f->d_ye, s, nullptr, true));
  FEM_TRY(fem_launch_scatter(L.f, FEM_F64, L.f->d_ye, y, L.f->d_ess_mask, x, nullptr, 0, s, nullptr, true));
  k_resid<<<m->nb, 256, 0, s>>>(L.n, b, y, r, m->part);
  k_sum1<<<1, kRed, 0, s>>>(m->part, m->nb, m->part + 3 * m->nb);
  FEM_LAUNCHED();
  return read_words(m, m->part + 3 * m->nb, sizeof(double), rr, s);
}

}  // namespace

extern "C" fem_status fem_mg_solve(fem_mg* m, const double* b, double* xio, const fem_solve_opts* opts,
                                   fem_solve_info* info, void* stream) {
  if (!m || !b || !xio) return fem_fail(FEM_EINVAL, "fem_mg_solve: NULL argument");
  fem_solve_opts o;
  fem_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0) || o.maxit <= 0) return fem_fail(FEM_EINVAL, "fem_mg_solve: rtol > 0 and maxit > 0 required");
  if (o.precision != FEM_SOLVE_F64 && o.precision != FEM_SOLVE_DF64 && o.precision != FEM_SOLVE_MIXED)
    return fem_fail(FEM_EINVAL, "fem_mg_solve: precision must be FEM_SOLVE_F64, FEM_SOLVE_DF64 or FEM_SOLVE_MIXED");
  const bool mixed = o.precision == FEM_SOLVE_MIXED;
  o.inner_rtol = fem_inner_rtol(o, 1);
  if (mixed && !(o.inner_rtol < 1.0))
    return fem_fail(FEM_EINVAL, "fem_mg_solve: FEM_SOLVE_MIXED needs inner_rtol < 1");
  const int dtype = o.precision == FEM_SOLVE_DF64 ? FEM_DF64 : mixed ? FEM_F32 : FEM_F64;
  cudaStream_t s = (cudaStream_t)stream;
  const MgLevel& L = m->lv[0];
  const int64_t n = L.n;
  if (dtype == FEM_DF64) FEM_TRY(fem_form_ensure_df64(L.f, s));
  if (mixed) {
    FEM_TRY(fem_form_ensure_f32(L.f, s));
    if (!m->w32) FEM_TRY(dev_alloc(&m->w32, (size_t)2 * n));
  }
  const int nb = m->nb;
  double* w = m->w64;
  double *x = w, *r = w + n, *rold = w + 2 * n, *z = w + 3 * n, *p = w + 4 * n, *q = w + 5 * n, *t = w + 6 * n;
  fem_solve_info inf;
  std::memset(&inf, 0, sizeof inf);
  FEM_CUDA(cudaMemcpyAsync(x, xio, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  // A_c x = b fixes the essential entries: x_ess = b_ess (the V-cycle never
  // corrects them, so an initial guess that disagrees there is replaced)
  k_copy_ess<<<vblocks(n), 256, 0, s>>>(n, L.f->d_ess_mask, b, x);
  FEM_LAUNCHED();
  // ||b||^2
  k_dot2<<<nb, 256, 0, s>>>(n, b, b, m->part);
  k_sum1<<<1, kRed, 0, s>>>(m->part, nb, m->part + 3 * nb);
  FEM_LAUNCHED();
  double bb = 0.0;
  FEM_TRY(read_words(m, m->part + 3 * nb, sizeof(double), &bb, s));
  inf.bnorm = std::sqrt(bb);
  if (!std::isfinite(bb)) {
    if (info) *info = inf;
    return fem_fail(FEM_EBREAKDOWN, "fem_mg_solve: non-finite right-hand side");
  }
  if (!(bb > 0)) {
    FEM_CUDA(cudaMemsetAsync(xio, 0, sizeof(double) * n, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    inf.converged = 1;
    if (info) *info = inf;
    return FEM_OK;
  }
  const double tol2 = o.rtol * o.rtol * bb;
  const int k = o.check_every > 0 ? o.check_every : 4;
  int total = 0, restarts = 0, status = MS_NOCONV;
  double rr = 0.0;
  for (;;) {
    FEM_TRY(fine_residual(m, b, x, r, t, q, &rr, s));
    if (!std::isfinite(rr)) {
      status = MS_BREAK;
      break;
    }
    if (rr <= tol2) {
      status = MS_CONV;
      break;
    }
    if (total >= o.maxit || restarts > o.max_outer) {
      status = MS_NOCONV;
      break;
    }
    // z = M r, p = z, scalars
    FEM_TRY(precond(m, r, z, m->d_never, s));
    FEM_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    k_dot2<<<nb, 256, 0, s>>>(n, r, z, m->part);  // (r.z, r.r)
    // FP32 outer operator: each pass reduces the true residual by inner_rtol
    // (iterative refinement through the restarts); else straight to rtol
    const double tol_pass = mixed ? std::max(tol2, o.inner_rtol * o.inner_rtol * rr) : tol2;
    k_fg_init<<<1, kRed, 0, s>>>(m->sc, m->part, nb, tol_pass, o.maxit - total);
    FEM_LAUNCHED();
    // iterate: graph of k outer iterations, host polls between replays
    cudaGraphExec_t exec = nullptr;
    if (o.use_graph) {
      cudaStream_t cs;
      FEM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      fem_status st = FEM_OK;
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = fem_fail(FEM_ECUDA, "fem_mg_solve: capture failed to begin");
      } else {
        for (int i = 0; i < k && st == FEM_OK; ++i) st = fcg_iteration(m, dtype, x, r, rold, z, p, q, cs);
        const cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (st == FEM_OK && e != cudaSuccess) st = fem_fail(FEM_ECUDA, "fem_mg_solve: end capture failed");
      }
      if (st == FEM_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess)
        st = fem_fail(FEM_ECUDA, "fem_mg_solve: graph instantiation failed");
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      if (st != FEM_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        return st;
      }
    }
    fem_status st = FEM_OK;
    int words[4] = {0, 0, 0, 0};
    const int rounds = (o.maxit - total) / k + 2;
    for (int round = 0; round < rounds && st == FEM_OK; ++round) {
      if (exec) {
        if (cudaGraphLaunch(exec, s) != cudaSuccess) st = fem_fail(FEM_ECUDA, "fem_mg_solve: graph launch failed");
      } else {
        for (int i = 0; i < k && st == FEM_OK; ++i) st = fcg_iteration(m, dtype, x, r, rold, z, p, q, s);
      }
      if (st == FEM_OK) st = read_words(m, &m->sc->it, sizeof words, words, s);
      if (st == FEM_OK && words[1]) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (st != FEM_OK) return st;
    total += words[0];
    restarts += 1;
    if (!words[1] || words[2] == MS_NOCONV) {
      FEM_TRY(fine_residual(m, b, x, r, t, q, &rr, s));
      status = rr <= tol2 ? MS_CONV : MS_NOCONV;
      break;
    }
    if (words[2] == MS_BREAK) {
      FEM_TRY(fine_residual(m, b, x, r, t, q, &rr, s));
      status = rr <= tol2 ? MS_CONV : MS_BREAK;
      break;
    }
    // MS_CONV on the recursive residual: the loop head confirms with the true one
  }
  FEM_CUDA(cudaMemcpyAsync(xio, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  inf.iterations = total;
  inf.outer = restarts;
  inf.relres = std::sqrt(rr / bb);
  inf.converged = status == MS_CONV;
  if (info) *info = inf;
  if (status == MS_BREAK) return fem_fail(FEM_EBREAKDOWN, "fem_mg_solve: breakdown");
  if (status != MS_CONV)
    return fem_fail(FEM_ENOCONV, "fem_mg_solve: no convergence after %d iterations (relres %.3e)", total, inf.relres);
  return FEM_OK;
}
