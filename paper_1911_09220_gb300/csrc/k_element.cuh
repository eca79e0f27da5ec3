// Sum-factorized element operators shared by the standalone element kernels
// (k_apply.cu) and the persistent batched kernel (k_batch.cu).
//
// One element is handled by a (Q x Q) plane of threads (tx, ty); thread
// (qx, qy) owns a column of points along z. Contractions along x and y go
// through the plane's shared-memory slab `s` (Smem<D1,Q>::SE values), those
// along z run in registers:
//   gather   X[z][y][x]          = x_L[map[z][y][x]]              (G)
//   stage 1  BX, GX  [z][y][qx]  = sum_x B/G[qx][x] X              (B, x)
//   stage 2  bb, gb, bg [z]      = sum_y B/G[qy][y] (BX|GX)        (B, y)
//   stage 3  grad_q              = sum_z B/G[qz][z] (...)          (B, z)
//   point    v_q = D_q grad_q (D symmetric, 6 components)           (D)
//   back z   t0,t1,t2 [dz]      += B/G[qz][dz] v                  (B^T, z)
//   back y   UA, UB [dz][dy][qx] = sum_qy B/G[qy][dy] t            (B^T, y)
//   back x   Y[dz][dy][dx]       = sum_qx G[qx][dx] UA + B[qx][dx] UB
// (Sec. 4.4: B_ki = B1d_{k1 i1} B1d_{k2 i2} B1d_{k3 i3}, one direction at a
// time, O(p^{d+1}) operations per element.) Every thread of the block must
// call these functions the same number of times (they contain
// __syncthreads); threads of planes without an element pass valid = false
// and still own an in-bounds slab.
#pragma once

#include <stdint.h>

#include "k_df64.cuh"

template <int D1, int Q>
struct Smem {
  static constexpr int ND = D1 * D1 * D1;
  static constexpr int SA = ND + 2 * D1 * D1 * Q;          // X, BX, GX
  static constexpr int SB = 3 * D1 * Q * Q + 2 * D1 * D1 * Q;  // t0..t2, UA, UB
  static constexpr int SE = SA > SB ? SA : SB;             // per element, in T
};

// map: the element's DOF list (e2l + e*(p+1)^3); De: its D block
// (D + e*6*q^3); out: its E-vector slice. sB/sG: [Q][D1] tables in smem,
// written before the call. Dereferenced only when valid.
// T: compute type (double, float or df64); TX: type of x and out.
template <typename T, int D1, int Q, typename TX = T>
__device__ __forceinline__ void diffusion_element(int tx, int ty, bool valid, const int32_t* __restrict__ map,
                                                  const T* __restrict__ De, const T* sB, const T* sG, T* s,
                                                  const TX* __restrict__ x, TX* __restrict__ out) {
  constexpr int ND = D1 * D1 * D1, NQ = Q * Q * Q;
  T* sX = s;
  T* sBX = s + ND;
  T* sGX = sBX + D1 * D1 * Q;
  if (valid && tx < D1 && ty < D1) {
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      const int k = (z * D1 + ty) * D1 + tx;
      sX[k] = fe_from<T>(__ldg(x + __ldg(map + k)));
    }
  }
  __syncthreads();
  if (ty < D1) {  // stage 1: threads (qx, dy)
    T b[D1], g[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      b[d] = sB[tx * D1 + d];
      g[d] = sG[tx * D1 + d];
    }
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      T u = 0, v = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) {
        const T xv = sX[(z * D1 + ty) * D1 + d];
        u += b[d] * xv;
        v += g[d] * xv;
      }
      sBX[(z * D1 + ty) * Q + tx] = fe_norm(u);
      sGX[(z * D1 + ty) * Q + tx] = fe_norm(v);
    }
  }
  __syncthreads();
  T rbb[D1], rgb[D1], rbg[D1];
  {  // stage 2: threads (qx, qy)
    T b[D1], g[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      b[d] = sB[ty * D1 + d];
      g[d] = sG[ty * D1 + d];
    }
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      T bb = 0, gb = 0, bg = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) {
        const T u = sBX[(z * D1 + d) * Q + tx];
        const T v = sGX[(z * D1 + d) * Q + tx];
        bb += b[d] * u;
        gb += b[d] * v;
        bg += g[d] * u;
      }
      rbb[z] = fe_norm(bb);
      rgb[z] = fe_norm(gb);
      rbg[z] = fe_norm(bg);
    }
  }
  T t0[D1], t1[D1], t2[D1];
#pragma unroll
  for (int d = 0; d < D1; ++d) t0[d] = t1[d] = t2[d] = 0;
  const T* Dp = De + ty * Q + tx;
#pragma unroll 2
  for (int qz = 0; qz < Q; ++qz) {
    T g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      const T bz = sB[qz * D1 + z], gz = sG[qz * D1 + z];
      g0 += bz * rgb[z];
      g1 += bz * rbg[z];
      g2 += gz * rbb[z];
    }
    g0 = fe_norm(g0);
    g1 = fe_norm(g1);
    g2 = fe_norm(g2);
    const int o = qz * Q * Q;
    T d00 = 0, d01 = 0, d02 = 0, d11 = 0, d12 = 0, d22 = 0;
    if (valid) {
      d00 = fe_ldg(Dp + 0 * NQ + o);
      d01 = fe_ldg(Dp + 1 * NQ + o);
      d02 = fe_ldg(Dp + 2 * NQ + o);
      d11 = fe_ldg(Dp + 3 * NQ + o);
      d12 = fe_ldg(Dp + 4 * NQ + o);
      d22 = fe_ldg(Dp + 5 * NQ + o);
    }
    const T v0 = fe_norm(d00 * g0 + d01 * g1 + d02 * g2);
    const T v1 = fe_norm(d01 * g0 + d11 * g1 + d12 * g2);
    const T v2 = fe_norm(d02 * g0 + d12 * g1 + d22 * g2);
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      const T bz = sB[qz * D1 + d], gz = sG[qz * D1 + d];
      t0[d] += bz * v0;
      t1[d] += bz * v1;
      t2[d] += gz * v2;
    }
  }
  __syncthreads();  // phase-A buffers are dead from here on
  T* sT0 = s;
  T* sT1 = sT0 + D1 * Q * Q;
  T* sT2 = sT1 + D1 * Q * Q;
  T* sUA = sT2 + D1 * Q * Q;
  T* sUB = sUA + D1 * D1 * Q;
#pragma unroll
  for (int d = 0; d < D1; ++d) {
    const int k = (d * Q + ty) * Q + tx;
    sT0[k] = fe_norm(t0[d]);
    sT1[k] = fe_norm(t1[d]);
    sT2[k] = fe_norm(t2[d]);
  }
  __syncthreads();
  if (ty < D1) {  // back y: threads (qx, dy)
    T b[Q], g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      b[q] = sB[q * D1 + ty];
      g[q] = sG[q * D1 + ty];
    }
#pragma unroll
    for (int dz = 0; dz < D1; ++dz) {
      T ua = 0, ub = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = (dz * Q + q) * Q + tx;
        ua += b[q] * sT0[k];
        ub += g[q] * sT1[k] + b[q] * sT2[k];
      }
      sUA[(dz * D1 + ty) * Q + tx] = fe_norm(ua);
      sUB[(dz * D1 + ty) * Q + tx] = fe_norm(ub);
    }
  }
  __syncthreads();
  if (valid && tx < D1 && ty < D1) {  // back x: threads (dx, dy)
    T b[Q], g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      b[q] = sB[q * D1 + tx];
      g[q] = sG[q * D1 + tx];
    }
#pragma unroll
    for (int dz = 0; dz < D1; ++dz) {
      T y = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = (dz * D1 + ty) * Q + q;
        y += g[q] * sUA[k] + b[q] * sUB[k];
      }
      fe_store(&out[(dz * D1 + ty) * D1 + tx], y);
    }
  }
}

// Mass: the same passes with B only and one scalar D per point
// (Sec. 4.4, M_E = B^T D_E B). De: the element's D block (D + e*q^3).
template <typename T, int D1, int Q, typename TX = T>
__device__ __forceinline__ void mass_element(int tx, int ty, bool valid, const int32_t* __restrict__ map,
                                             const T* __restrict__ De, const T* sB, T* s,
                                             const TX* __restrict__ x, TX* __restrict__ out) {
  constexpr int ND = D1 * D1 * D1;
  T* sX = s;
  T* sBX = s + ND;
  if (valid && tx < D1 && ty < D1) {
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      const int k = (z * D1 + ty) * D1 + tx;
      sX[k] = fe_from<T>(__ldg(x + __ldg(map + k)));
    }
  }
  __syncthreads();
  if (ty < D1) {
    T b[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) b[d] = sB[tx * D1 + d];
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      T u = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) u += b[d] * sX[(z * D1 + ty) * D1 + d];
      sBX[(z * D1 + ty) * Q + tx] = fe_norm(u);
    }
  }
  __syncthreads();
  T rbb[D1];
  {
    T b[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) b[d] = sB[ty * D1 + d];
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      T bb = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) bb += b[d] * sBX[(z * D1 + d) * Q + tx];
      rbb[z] = fe_norm(bb);
    }
  }
  T t0[D1];
#pragma unroll
  for (int d = 0; d < D1; ++d) t0[d] = 0;
  const T* Dp = De + ty * Q + tx;
#pragma unroll 2
  for (int qz = 0; qz < Q; ++qz) {
    T u = 0;
#pragma unroll
    for (int z = 0; z < D1; ++z) u += sB[qz * D1 + z] * rbb[z];
    const T v = valid ? fe_ldg(Dp + qz * Q * Q) * fe_norm(u) : T(0);
#pragma unroll
    for (int d = 0; d < D1; ++d) t0[d] += sB[qz * D1 + d] * v;
  }
  __syncthreads();
  T* sT0 = s;
  T* sUA = sT0 + D1 * Q * Q;
#pragma unroll
  for (int d = 0; d < D1; ++d) sT0[(d * Q + ty) * Q + tx] = fe_norm(t0[d]);
  __syncthreads();
  if (ty < D1) {
    T b[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) b[q] = sB[q * D1 + ty];
#pragma unroll
    for (int dz = 0; dz < D1; ++dz) {
      T ua = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) ua += b[q] * sT0[(dz * Q + q) * Q + tx];
      sUA[(dz * D1 + ty) * Q + tx] = fe_norm(ua);
    }
  }
  __syncthreads();
  if (valid && tx < D1 && ty < D1) {
    T b[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) b[q] = sB[q * D1 + tx];
#pragma unroll
    for (int dz = 0; dz < D1; ++dz) {
      T y = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) y += b[q] * sUA[(dz * D1 + ty) * Q + q];
      fe_store(&out[(dz * D1 + ty) * D1 + tx], y);
    }
  }
}

