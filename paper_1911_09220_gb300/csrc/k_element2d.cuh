// The quadrilateral (2D) element operator y_e = G^T B^T D B G x_e as a block
// driver shared by the 2D element kernel (k_2d.cu) and the batched kernel
// (k_batch.cu). Sum factorization in two directions (Sec. 4.4 with d = 2),
// one element per row of Q threads (index t):
//   gather X[y][x] = x_L[map[y][x]]
//   S1 (y lines):  BX, GX[qx][y] = sum_x B/G[qx][x] X[y][x]
//   S2 (qx lines): grad at (qx, qy): g0 = sum_y B[qy][y] GX, g1 = sum_y G[qy][y] BX;
//                  v = D_q g; back along y: T0 = B^T_y v0, T1 = G^T_y v1
//   S3 (dy lines): Y[dy][dx] = sum_qx G[qx][dx] T0 + B[qx][dx] T1
// Every line goes through the even-odd form of its 1D operator with folded
// coefficients from constant memory (k_tables.cuh), as in 3D.
#pragma once

#include "k_element.cuh"

template <int D1, int Q>
struct Smem2 {
  static constexpr int XP = D1 | 1;  // padded x rows of X
  static constexpr int YP = D1 | 1;  // padded y rows of BX, GX
  static constexpr int QP = Q | 1;   // padded qx rows of T0, T1
  static constexpr int SE = D1 * XP + 2 * Q * YP + 2 * D1 * QP;  // per element, in T
};

// Elements per block: rows of Q threads, about 128 threads per block.
__host__ __device__ constexpr int ne2(int Q) { return Q <= 3 ? 42 : Q <= 4 ? 32 : Q <= 6 ? 21 : Q <= 8 ? 16 : 12; }

// Element rows el of the block (thread (t, el), t < Q) work on elements
// e0 + el for el < nel; the others take part with valid = false and still
// own a slab of Smem2<D1, Q>::SE values. Element e's DOF list is
// e2l + e * D1^2, its D block Dq + e * NC * Q^2; the output goes to the
// element-major E-vector ye + e * D1^2, or (pos given) to ye[pos[e * D1^2 +
// k]], the DOF-sorted order. Every thread of the block must call it (it
// contains __syncthreads).
template <typename T, int D1, int Q, typename TX, bool DIFF>
__device__ __forceinline__ void quad_block(int t, int el, int64_t e0, int nel, const int32_t* __restrict__ e2l,
                                           const T* __restrict__ Dq, T* sm, const TX* __restrict__ x,
                                           TX* __restrict__ ye, const int32_t* __restrict__ pos = nullptr) {
  using L = Smem2<D1, Q>;
  constexpr int XP = L::XP, YP = L::YP, QP = L::QP, ND = D1 * D1, NQ = Q * Q;
  constexpr int BF = eo_off(D1, Q, 0), GF = eo_off(D1, Q, 1), BT = eo_off(D1, Q, 2), GT = eo_off(D1, Q, 3);
  // slab offsets: X [y][XP], BX, GX [qx][YP], T0, T1 [dy][QP]
  constexpr int OBX = D1 * XP, OGX = OBX + Q * YP, OT0 = OGX + Q * YP, OT1 = OT0 + D1 * QP;
  const int tid = t + Q * el;
  const bool valid = el < nel;
  const int64_t e = valid ? e0 + el : 0;
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
    const int64_t oo = (e0 + el3) * ND + t * D1;  // element-major slot of (element, line)
    if constexpr (DIFF) {
      T a1[Q], y2[D1];
#pragma unroll
      for (int q = 0; q < Q; ++q) a1[q] = sT1[t * QP + q];
      eo_line<T, D1, Q, -1, GT>(a0, y1);
      eo_line<T, D1, Q, 1, BT>(a1, y2);
#pragma unroll
      for (int dx = 0; dx < D1; ++dx) fe_store(ye + (pos ? (int64_t)__ldg(pos + oo + dx) : oo + dx), y1[dx] + y2[dx]);
    } else {
      eo_line<T, D1, Q, 1, BT>(a0, y1);
#pragma unroll
      for (int dx = 0; dx < D1; ++dx) fe_store(ye + (pos ? (int64_t)__ldg(pos + oo + dx) : oo + dx), y1[dx]);
    }
  }
}
