// Sum-factorized element operators shared by the standalone element kernels
// (k_apply.cu) and the persistent batched kernel (k_batch.cu).
//
// The operator is y_e = G_e^T B^T D_e B G_e x (Sec. 4.3) with the basis
// evaluator applied one direction at a time (Sec. 4.4: B_ki = B1d_{k1 i1}
// B1d_{k2 i2} B1d_{k3 i3}, O(p^{d+1}) operations per element).
//
// One element is handled by a plane of Q*Q threads (index t). Every
// contraction stage gives each active thread one *line* of its input tensor:
// the thread reads the line (K values) from shared memory into registers and
// produces every output of that line (M values), so each loaded value feeds
// M (or 2M, 3M) FMAs. The 1D coefficients come from constant memory at
// compile-time indices (k_tables.cuh): they are FMA operands, not loads.
//   gather  X[z][y][x]           = x_L[map[z][y][x]]                   (G)
//   S1  (z, y) lines:  BX, GX[z][qx][y] = sum_x B/G[qx][x] X[z][y][x]   (x)
//   S2  (z, qx) lines: BB, GB, BG[z][qy][qx] = sum_y B/G[qy][y] (BX|GX) (y)
//   S3  (qy, qx) lines: grad at (qz,qy,qx) = sum_z B/G[qz][z] (..)      (z)
//       D: v = D_q grad (6 symmetric components) at every qz            (D)
//       back z: T0, T1, T2[dz][qy][qx] = sum_qz B/G[qz][dz] v           (z^T)
//   S4  (dz, qx) lines: UA, UB[dz][dy][qx] = sum_qy B/G[qy][dy] T       (y^T)
//   S5  (dz, dy) lines: Y[dz][dy][dx] = sum_qx G[qx][dx] UA + B[qx][dx] UB (x^T)
// Rows that threads read along are padded to an odd length so that lines of
// neighbouring threads fall in different shared-memory banks.
//
// Every thread of the block must call these functions the same number of
// times (they contain __syncthreads); a plane without an element passes
// valid = false and still owns an in-bounds slab of ElemSmem<D1,Q>::SE values.
#pragma once

#include <stdint.h>

#include "k_df64.cuh"
#include "k_tables.cuh"

template <int D1, int Q>
struct ElemSmem {
  static constexpr int XP = D1 | 1;  // padded x rows of X
  static constexpr int YP = D1 | 1;  // padded y rows of BX, GX
  static constexpr int QP = Q | 1;   // padded qx rows of UA, UB
  static constexpr int SA = D1 * D1 * XP + 2 * D1 * Q * YP + 3 * D1 * Q * Q;
  static constexpr int SB = 3 * D1 * Q * Q + 2 * D1 * D1 * QP;
  static constexpr int SE = SA > SB ? SA : SB;  // per element, in T
};

// map: the element's DOF list (e2l + e*(p+1)^3); De: its D block
// (D + e*6*q^3); out: its E-vector slice. Dereferenced only when valid.
// T: compute type (double, float or df64); TX: type of x and out.
template <typename T, int D1, int Q, typename TX = T>
__device__ __forceinline__ void diffusion_element(int t, bool valid, const int32_t* __restrict__ map,
                                                  const T* __restrict__ De, T* s, const TX* __restrict__ x,
                                                  TX* __restrict__ out) {
  using L = ElemSmem<D1, Q>;
  constexpr int ND = D1 * D1 * D1, NQ = Q * Q * Q, QQ = Q * Q, XP = L::XP, YP = L::YP, QP = L::QP;
  constexpr int OFF = tab_off(D1, Q);
  T* sX = s;                                // [z][y][XP]
  T* sBX = sX + D1 * D1 * XP;               // [z][qx][YP]
  T* sGX = sBX + D1 * Q * YP;
  T* sBB = sGX + D1 * Q * YP;               // [z][qy][qx]
  T* sGB = sBB + D1 * QQ;
  T* sBG = sGB + D1 * QQ;
  if (valid) {
    for (int k = t; k < ND; k += QQ) {
      const int xi = k % D1, row = k / D1;
      sX[row * XP + xi] = fe_from<T>(__ldg(x + __ldg(map + k)));
    }
  }
  __syncthreads();
  if (t < D1 * D1) {  // S1: line (z, y) along x
    const int z = t / D1, y = t % D1;
    T xr[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) xr[d] = sX[t * XP + d];
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) {
      T u = 0, v = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) {
        u += Tab<T>::B(OFF + qx * D1 + d) * xr[d];
        v += Tab<T>::G(OFF + qx * D1 + d) * xr[d];
      }
      sBX[(z * Q + qx) * YP + y] = fe_norm(u);
      sGX[(z * Q + qx) * YP + y] = fe_norm(v);
    }
  }
  __syncthreads();
  if (t < D1 * Q) {  // S2: line (z, qx) along y
    const int z = t / Q, qx = t % Q;
    T br[D1], gr[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      br[d] = sBX[t * YP + d];
      gr[d] = sGX[t * YP + d];
    }
#pragma unroll
    for (int qy = 0; qy < Q; ++qy) {
      T bb = 0, gb = 0, bg = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) {
        const T b = Tab<T>::B(OFF + qy * D1 + d);
        bb += b * br[d];
        gb += b * gr[d];
        bg += Tab<T>::G(OFF + qy * D1 + d) * br[d];
      }
      const int o = (z * Q + qy) * Q + qx;
      sBB[o] = fe_norm(bb);
      sGB[o] = fe_norm(gb);
      sBG[o] = fe_norm(bg);
    }
  }
  __syncthreads();
  T t0[D1], t1[D1], t2[D1];
#pragma unroll
  for (int d = 0; d < D1; ++d) t0[d] = t1[d] = t2[d] = 0;
  if (t < QQ) {  // S3: line (qy, qx) along z, D at every point, back along z
    T rbb[D1], rgb[D1], rbg[D1];
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      rbb[z] = sBB[z * QQ + t];
      rgb[z] = sGB[z * QQ + t];
      rbg[z] = sBG[z * QQ + t];
    }
    const T* Dp = De + t;
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) {
      T g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
      for (int z = 0; z < D1; ++z) {
        const T b = Tab<T>::B(OFF + qz * D1 + z);
        g0 += b * rgb[z];
        g1 += b * rbg[z];
        g2 += Tab<T>::G(OFF + qz * D1 + z) * rbb[z];
      }
      g0 = fe_norm(g0);
      g1 = fe_norm(g1);
      g2 = fe_norm(g2);
      const int o = qz * QQ;
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
        const T b = Tab<T>::B(OFF + qz * D1 + d);
        t0[d] += b * v0;
        t1[d] += b * v1;
        t2[d] += Tab<T>::G(OFF + qz * D1 + d) * v2;
      }
    }
  }
  __syncthreads();  // phase-A arrays are dead from here on
  T* sT0 = s;                               // [dz][qy][qx]
  T* sT1 = sT0 + D1 * QQ;
  T* sT2 = sT1 + D1 * QQ;
  T* sUA = sT2 + D1 * QQ;                   // [dz][dy][QP]
  T* sUB = sUA + D1 * D1 * QP;
  if (t < QQ) {
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      sT0[d * QQ + t] = fe_norm(t0[d]);
      sT1[d * QQ + t] = fe_norm(t1[d]);
      sT2[d * QQ + t] = fe_norm(t2[d]);
    }
  }
  __syncthreads();
  if (t < D1 * Q) {  // S4: line (dz, qx) along qy
    const int dz = t / Q, qx = t % Q;
    T a0[Q], a1[Q], a2[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int o = (dz * Q + q) * Q + qx;
      a0[q] = sT0[o];
      a1[q] = sT1[o];
      a2[q] = sT2[o];
    }
#pragma unroll
    for (int dy = 0; dy < D1; ++dy) {
      T ua = 0, ub = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const T b = Tab<T>::B(OFF + q * D1 + dy);
        ua += b * a0[q];
        ub += Tab<T>::G(OFF + q * D1 + dy) * a1[q];
        ub += b * a2[q];
      }
      sUA[(dz * D1 + dy) * QP + qx] = fe_norm(ua);
      sUB[(dz * D1 + dy) * QP + qx] = fe_norm(ub);
    }
  }
  __syncthreads();
  if (valid && t < D1 * D1) {  // S5: line (dz, dy) along qx
    T ua[Q], ub[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      ua[q] = sUA[t * QP + q];
      ub[q] = sUB[t * QP + q];
    }
#pragma unroll
    for (int dx = 0; dx < D1; ++dx) {
      T y = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        y += Tab<T>::G(OFF + q * D1 + dx) * ua[q];
        y += Tab<T>::B(OFF + q * D1 + dx) * ub[q];
      }
      fe_store(&out[t * D1 + dx], y);
    }
  }
}

// Mass: the same lines with B only and one scalar D per point
// (Sec. 4.4, M_E = B^T D_E B). De: the element's D block (D + e*q^3).
template <typename T, int D1, int Q, typename TX = T>
__device__ __forceinline__ void mass_element(int t, bool valid, const int32_t* __restrict__ map,
                                             const T* __restrict__ De, T* s, const TX* __restrict__ x,
                                             TX* __restrict__ out) {
  using L = ElemSmem<D1, Q>;
  constexpr int ND = D1 * D1 * D1, QQ = Q * Q, XP = L::XP, YP = L::YP, QP = L::QP;
  constexpr int OFF = tab_off(D1, Q);
  T* sX = s;
  T* sBX = sX + D1 * D1 * XP;
  T* sBB = sBX + D1 * Q * YP;
  if (valid) {
    for (int k = t; k < ND; k += QQ) {
      const int xi = k % D1, row = k / D1;
      sX[row * XP + xi] = fe_from<T>(__ldg(x + __ldg(map + k)));
    }
  }
  __syncthreads();
  if (t < D1 * D1) {
    const int z = t / D1, y = t % D1;
    T xr[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) xr[d] = sX[t * XP + d];
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) {
      T u = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) u += Tab<T>::B(OFF + qx * D1 + d) * xr[d];
      sBX[(z * Q + qx) * YP + y] = fe_norm(u);
    }
  }
  __syncthreads();
  if (t < D1 * Q) {
    const int z = t / Q, qx = t % Q;
    T br[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) br[d] = sBX[t * YP + d];
#pragma unroll
    for (int qy = 0; qy < Q; ++qy) {
      T bb = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) bb += Tab<T>::B(OFF + qy * D1 + d) * br[d];
      sBB[(z * Q + qy) * Q + qx] = fe_norm(bb);
    }
  }
  __syncthreads();
  T t0[D1];
#pragma unroll
  for (int d = 0; d < D1; ++d) t0[d] = 0;
  if (t < QQ) {
    T rbb[D1];
#pragma unroll
    for (int z = 0; z < D1; ++z) rbb[z] = sBB[z * QQ + t];
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) {
      T u = 0;
#pragma unroll
      for (int z = 0; z < D1; ++z) u += Tab<T>::B(OFF + qz * D1 + z) * rbb[z];
      const T v = valid ? fe_ldg(De + t + qz * QQ) * fe_norm(u) : T(0);
      const T vn = fe_norm(v);
#pragma unroll
      for (int d = 0; d < D1; ++d) t0[d] += Tab<T>::B(OFF + qz * D1 + d) * vn;
    }
  }
  __syncthreads();
  T* sT0 = s;
  T* sUA = sT0 + D1 * QQ;
  if (t < QQ) {
#pragma unroll
    for (int d = 0; d < D1; ++d) sT0[d * QQ + t] = fe_norm(t0[d]);
  }
  __syncthreads();
  if (t < D1 * Q) {
    const int dz = t / Q, qx = t % Q;
    T a0[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) a0[q] = sT0[(dz * Q + q) * Q + qx];
#pragma unroll
    for (int dy = 0; dy < D1; ++dy) {
      T ua = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) ua += Tab<T>::B(OFF + q * D1 + dy) * a0[q];
      sUA[(dz * D1 + dy) * QP + qx] = fe_norm(ua);
    }
  }
  __syncthreads();
  if (valid && t < D1 * D1) {
    T ua[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) ua[q] = sUA[t * QP + q];
#pragma unroll
    for (int dx = 0; dx < D1; ++dx) {
      T y = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) y += Tab<T>::B(OFF + q * D1 + dx) * ua[q];
      fe_store(&out[t * D1 + dx], y);
    }
  }
}

// Hint the L2 to fetch a contiguous byte range with one bulk prefetch
// (cp.async.bulk.prefetch.L2: no completion to wait for). The range is
// trimmed to 16-byte boundaries as the instruction requires.
__device__ __forceinline__ void l2_prefetch_range(const void* p, size_t bytes) {
  const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
  const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes) & ~(uintptr_t)15;
  if (e > a) {
    const unsigned n = (unsigned)(e - a);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
  }
}
