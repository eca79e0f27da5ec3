// Sum-factorized element operators shared by the standalone element kernels
// (k_apply.cu) and the persistent batched kernel (k_batch.cu).
//
// The operator is y_e = G_e^T B^T D_e B G_e x (Sec. 4.3) with the basis
// evaluator applied one direction at a time (Sec. 4.4: B_ki = B1d_{k1 i1}
// B1d_{k2 i2} B1d_{k3 i3}, O(p^{d+1}) operations per element).
//
// Every contraction stage gives each active thread one *line* of its input
// tensor (the drivers at the end of this file decide which thread runs
// which line of which element):
// the thread reads the line (K values) from shared memory into registers and
// produces every output of that line (M values), so each loaded value feeds
// many FMAs. Each line goes through the even-odd (folded) form of its 1D
// operator (eo_apply below), and the folded coefficients come from constant
// memory at compile-time indices (k_tables.cuh): they are FMA operands, not
// loads.
//   gather  X[z][y][x]           = x_L[map[z][y][x]]                   (G)
//   S1  (z, y) lines:  BX, GX[z][qx][y] = sum_x B/G[qx][x] X[z][y][x]   (x)
//   S2  (z, qx) lines: BB, GB, BG[z][qy][qx] = sum_y B/G[qy][y] (BX|GX) (y)
//   S3  (qy, qx) lines: grad at (qz,qy,qx) = sum_z B/G[qz][z] (..)      (z)
//       D: v = D_q grad (6 symmetric components) at every qz            (D)
//       back z: T0, T1, T2[dz][qy][qx] = sum_qz B/G[qz][dz] v           (z^T)
//   S4  (dz, qx) lines: UA, UB[dz][dy][qx] = sum_qy B/G[qy][dy] T       (y^T)
//   S5  (dz, dy) lines: Y[dz][dy][dx] = sum_qx G[qx][dx] UA + B[qx][dx] UB (x^T)
// Each stage's outputs are stored in its own thread order (consecutive words
// per store) with row strides searched at compile time against the next
// stage's read pattern (ElemSmem below), so that neither side of a stage
// boundary replays for bank conflicts.
//
// Every thread of the block must call the drivers the same number of times
// (they contain __syncthreads); a plane without an element passes valid =
// false and still owns an in-bounds slab of ElemSmem<T,D1,Q>::SE values.
#pragma once

#include <stdint.h>

#include <type_traits>

#include "k_df64.cuh"
#include "k_tables.cuh"

// ------------------------------------------------------------- even-odd ----
// One line through a folded 1D operator (k_tables.cuh): y[M] = A x[K], where
// e/o are the line's even and odd parts. P_k uses e, N_k uses o, and
// y_k = P_k + N_k, y_{M-1-k} = S (P_k - N_k): about half the multiply-adds
// of the plain M x K product.
template <typename T, int K>
__device__ __forceinline__ void eo_split(const T* x, T* e, T* o) {
#pragma unroll
  for (int j = 0; j < K / 2; ++j) {
    e[j] = fe_norm(x[j] + x[K - 1 - j]);
    o[j] = fe_norm(x[j] - x[K - 1 - j]);
  }
  if (K & 1) e[K / 2] = x[K / 2];
}

template <typename T, int M, int K, int S, int OFF>
__device__ __forceinline__ void eo_apply(const T* e, const T* o, T* y) {
  constexpr int hK = K / 2, cK = (K + 1) / 2, hM = M / 2, cM = (M + 1) / 2;
#pragma unroll
  for (int k = 0; k < cM; ++k) {
    const bool mid = (M & 1) && (k == hM);
    T P = 0, N = 0;
    if (!mid || S > 0) {
#pragma unroll
      for (int j = 0; j < cK; ++j) P += EO<T>::c(OFF + k * cK + j) * e[j];
    }
    if (!mid || S < 0) {
#pragma unroll
      for (int j = 0; j < hK; ++j) N += EO<T>::c(OFF + cM * cK + k * hK + j) * o[j];
    }
    if (mid) {
      y[k] = fe_norm(S > 0 ? P : N);
    } else {
      y[k] = fe_norm(P + N);
      y[M - 1 - k] = fe_norm(S > 0 ? P - N : N - P);
    }
  }
}

// y = A x for one line (split and apply).
template <typename T, int M, int K, int S, int OFF>
__device__ __forceinline__ void eo_line(const T* x, T* y) {
  T e[(K + 1) / 2], o[K / 2 > 0 ? K / 2 : 1];
  eo_split<T, K>(x, e, o);
  eo_apply<T, M, K, S, OFF>(e, o, y);
}

// The six D components of one point (point-major layout, 16-byte aligned
// for double and df64 records of 48 bytes, 8-byte aligned for float records
// of 24 bytes): three vector loads instead of six scalar ones.
__device__ __forceinline__ void d_load6(const double* p, double* d) {
  const double2* v = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double2 w = __ldg(v + k);
    d[2 * k] = w.x;
    d[2 * k + 1] = w.y;
  }
}
__device__ __forceinline__ void d_load6(const float* p, float* d) {
  const float2* v = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 w = __ldg(v + k);
    d[2 * k] = w.x;
    d[2 * k + 1] = w.y;
  }
}
__device__ __forceinline__ void d_load6(const df64* p, df64* d) {
  const float4* v = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 w = __ldg(v + k);
    d[2 * k] = df64(w.x, w.y);
    d[2 * k + 1] = df64(w.z, w.w);
  }
}

// The twelve values of one elasticity point record (J^-1 row-major, w det J
// lambda, w det J mu, pad): 96-byte records for double and double-float,
// 48-byte for float, loaded as 16-byte vectors.
__device__ __forceinline__ void d_load12(const double* p, double* d) {
  const double2* v = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double2 w = __ldg(v + k);
    d[2 * k] = w.x;
    d[2 * k + 1] = w.y;
  }
}
__device__ __forceinline__ void d_load12(const float* p, float* d) {
  const float4* v = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 w = __ldg(v + k);
    d[4 * k] = w.x;
    d[4 * k + 1] = w.y;
    d[4 * k + 2] = w.z;
    d[4 * k + 3] = w.w;
  }
}
__device__ __forceinline__ void d_load12(const df64* p, df64* d) {
  const float4* v = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 w = __ldg(v + k);
    d[2 * k] = df64(w.x, w.y);
    d[2 * k + 1] = df64(w.z, w.w);
  }
}

// Gather the element's DOF values x[map[k]] into the padded X rows: each
// thread first loads all its map entries, then all its x values, so the
// dependent load pairs of its ceil(D1^3 / Q^2) points are in flight together.
// (The FP64 kernel, bound by its arithmetic pipe, measured 1.2 % faster with
// the plain strided loop, which it keeps.)
template <typename T, int D1, int Q, typename TX>
__device__ __forceinline__ void gather_x(int t, bool valid, const int32_t* __restrict__ map,
                                         const TX* __restrict__ x, T* sX, int XP) {
  constexpr int ND = D1 * D1 * D1, QQ = Q * Q, NG = (ND + QQ - 1) / QQ;
  if constexpr (std::is_same<T, double>::value) {
    if (valid) {
      for (int k = t; k < ND; k += QQ) sX[(k / D1) * XP + k % D1] = fe_from<T>(__ldg(x + __ldg(map + k)));
    }
  } else {
    int32_t m[NG];
#pragma unroll
    for (int j = 0; j < NG; ++j) {
      const int k = t + j * QQ;
      m[j] = (valid && k < ND) ? __ldg(map + k) : -1;
    }
    TX v[NG];
#pragma unroll
    for (int j = 0; j < NG; ++j) v[j] = m[j] >= 0 ? __ldg(x + m[j]) : TX(0);
#pragma unroll
    for (int j = 0; j < NG; ++j) {
      const int k = t + j * QQ;
      if (m[j] >= 0) sX[(k / D1) * XP + k % D1] = fe_from<T>(v[j]);
    }
  }
}

// ------------------------------------------------ shared-memory strides ----
// Every intermediate tensor of the stages is stored in the order its writer
// threads produce it (writer r stores word row * S + r: consecutive words,
// no bank conflict), and its row stride S is chosen at compile time to
// minimise the bank conflicts of its reader threads. Reader r of n reads word
// (r % A) * m_lo + (r / A) * m_hi, with S in one of the two places. The cost
// of a candidate S splits the readers of one element into bank groups (32
// threads for 4-byte words; 16 for 8-byte words, which a warp accesses in two
// halves) and sums, over the groups, the largest number of threads whose
// words fall in one bank (distinct words, since every reader reads its own).
__host__ __device__ constexpr int bank_cost(int n, int A, int m_lo, int m_hi, int wbytes) {
  const int G = wbytes == 8 ? 16 : 32;
  int cost = 0;
  for (int g0 = 0; g0 < n; g0 += G) {
    int cnt[32] = {};
    int worst = 0;
    for (int r = g0; r < n && r < g0 + G; ++r) {
      const int w = (r % A) * m_lo + (r / A) * m_hi;
      const int b = w % G;
      cnt[b] += 1;
      if (cnt[b] > worst) worst = cnt[b];
    }
    cost += worst;
  }
  return cost;
}

// Smallest stride >= lo of least reader cost (candidates lo .. lo + 31).
__host__ __device__ constexpr int best_stride(int lo, int n, int A, bool stride_lo, int m_other, int wbytes) {
  int best = lo, best_cost = 1 << 30;
  for (int s = lo; s < lo + 32; ++s) {
    const int c = stride_lo ? bank_cost(n, A, s, m_other, wbytes) : bank_cost(n, A, m_other, s, wbytes);
    if (c < best_cost) {
      best_cost = c;
      best = s;
    }
  }
  return best;
}

// The same cost with the readers of NE consecutive elements side by side
// (reader i belongs to element i / L, whose slab starts SE words after the
// previous one; lanes n .. L-1 of an element are idle, L = n when the lines
// are packed): packed stages and the S3 planes put the lines of two elements
// into one warp whenever n is not a multiple of the bank group.
__host__ __device__ constexpr int bank_cost_packed(int n, int A, int m_lo, int m_hi, int wbytes, int ne, int se,
                                                   int L = 0) {
  const int G = wbytes == 8 ? 16 : 32;
  if (L < n) L = n;
  const int total = ne * L;
  int cost = 0;
  for (int g0 = 0; g0 < total; g0 += G) {
    int cnt[32] = {};
    int worst = 0;
    for (int i = g0; i < total && i < g0 + G; ++i) {
      const int el = i / L, r = i % L;
      if (r >= n) continue;
      const int w = el * se + (r % A) * m_lo + (r / A) * m_hi;
      const int b = w % G;
      cnt[b] += 1;
      if (cnt[b] > worst) worst = cnt[b];
    }
    cost += worst;
  }
  return cost;
}

// Lanes one element's lines take in a stage of n lines per element (the
// stages S1, S5: D1^2 lines; S2, S4: D1 q). FP32 blocks give each element
// its own half-warp or warp there when 8 < n <= 32 and its plane of QQ
// threads has that many lanes: then no warp of those stages touches two
// elements' slabs, whose relative bank offset no single slab stride can
// suit in all four stages at once (the buffer strides already make one
// element's lines conflict-free), and the slab stride only has to suit the
// S3 planes. In a bank model of every stage's accesses this removes the
// bank-conflict replays of the FP32 block at p = 4, q = 6 (30 % of its
// shared-memory wavefronts; p = 2, q = 4: 17 %); measured, the FP32 element
// kernel at p = 4 ran 10 % faster and at p = 2 3 % faster, while elements of
// two or more warps (p >= 5) gained nothing and keep the packed lines.
// FP64 and double-float blocks pack the lines of consecutive elements onto
// the lowest thread ids (L = n): an arithmetic-bound warp pays its issue
// slot however few lanes are active. (Build option FEM_F32_LANES=0 packs the
// FP32 stages too.)
#ifndef FEM_F32_LANES
#define FEM_F32_LANES 1
#endif
template <typename T>
__host__ __device__ constexpr int stage_lanes(int n, int QQ) {
  if (FEM_F32_LANES == 0 || !std::is_same<T, float>::value || n <= 8 || n > 32) return n;
  const int L = n <= 16 ? 16 : 32;
  return L <= QQ ? L : n;
}

// Slab stride >= lo (candidates lo .. lo + 31) of least total cost over the
// shared-memory accesses of all stages, each weighted by the values a line
// reads or writes (S1: X rows in, BX/GX out; S2: BX/GX in, BB/GB/BG out;
// S3: BB/GB/BG in, T0-T2 out; S4: T0-T2 in, UA/UB out; S5: UA/UB in),
// modelled on 8 elements whose S1/S5 lines take L1 lanes each and S2/S4
// lines L2 (stage_lanes).
__host__ __device__ constexpr int best_slab(int lo, int D1, int Q, int XP, int RB, int RC, int RT, int RU,
                                            int wbytes, int L1 = 0, int L2 = 0) {
  const int N1 = D1 * D1, N2 = D1 * Q, QQ = Q * Q, NEm = 8;
  int best = lo, best_cost = 1 << 30;
  for (int se = lo; se < lo + 32; ++se) {
    const int c = D1 * bank_cost_packed(N1, N1, XP, 0, wbytes, NEm, se, L1) +
                  2 * Q * bank_cost_packed(N1, N1, 1, 0, wbytes, NEm, se, L1) +
                  2 * D1 * bank_cost_packed(N2, Q, RB, D1, wbytes, NEm, se, L2) +
                  3 * Q * bank_cost_packed(N2, N2, 1, 0, wbytes, NEm, se, L2) +
                  3 * D1 * bank_cost_packed(QQ, Q, 1, RC, wbytes, NEm, se) +
                  3 * D1 * bank_cost_packed(QQ, QQ, 1, 0, wbytes, NEm, se) +
                  3 * Q * bank_cost_packed(N2, Q, 1, RT, wbytes, NEm, se, L2) +
                  2 * D1 * bank_cost_packed(N2, N2, 1, 0, wbytes, NEm, se, L2) +
                  2 * Q * bank_cost_packed(N1, D1, RU, Q, wbytes, NEm, se, L1);
    if (c < best_cost) {
      best_cost = c;
      best = se;
    }
  }
  return best;
}

// Per-element shared-memory plan (in units of T):
//   phase A  region 0: X [z][y][XP], dead after S1, then BB, GB, BG [qy][RC]
//            over (z, qx); region 1 (offset R0): BX, GX [qx][RB] over (z, y)
//   phase B  T0, T1, T2 [dz][RT] over (qy, qx);  UA, UB [dy][RU] over (dz, qx)
template <typename T, int D1, int Q>
struct ElemSmem {
  static constexpr int W = (int)sizeof(T);
  static constexpr int XP = D1 | 1;  // odd x rows: S1 reads rows with stride XP
  static constexpr int RB = best_stride(D1 * D1, D1 * Q, Q, true, D1, W);  // S2 reader (z, qx)
  static constexpr int RC = best_stride(D1 * Q, Q * Q, Q, false, 1, W);    // S3 reader (qy, qx)
  static constexpr int RT = best_stride(Q * Q, D1 * Q, Q, false, 1, W);    // S4 reader (dz, qx)
  static constexpr int RU = best_stride(D1 * Q, D1 * D1, D1, true, Q, W);  // S5 reader (dz, dy)
  static constexpr int R0 = D1 * D1 * XP > 3 * Q * RC ? D1 * D1 * XP : 3 * Q * RC;
  static constexpr int SA = R0 + 2 * Q * RB;
  static constexpr int SB = 3 * D1 * RT + 2 * D1 * RU;
  // lanes per element of the S1/S5 and S2/S4 lines (stage_lanes)
  static constexpr int L1 = stage_lanes<T>(D1 * D1, Q * Q);
  static constexpr int L2 = stage_lanes<T>(D1 * Q, Q * Q);
  // per element, in T: the larger phase, padded to the slab stride of least
  // bank conflicts between neighbouring elements' slabs (one slab per
  // element, the drivers' lane mapping)
  static constexpr int SE = best_slab(SA > SB ? SA : SB, D1, Q, XP, RB, RC, RT, RU, W, L1, L2);
  // the same for the elasticity block, whose stages pack the lines of its
  // (element, component) slabs (three per element) over all its threads
  static constexpr int SE3 = best_slab(SA > SB ? SA : SB, D1, Q, XP, RB, RC, RT, RU, W);
};

// ------------------------------------------------------ stage bodies ----
// One line of one stage on the slab s of one element (ElemSmem layout). The
// drivers below decide which thread runs which line of which element.
template <typename T, int D1, int Q>
struct Lines {
  using L = ElemSmem<T, D1, Q>;
  static constexpr int QQ = Q * Q, XP = L::XP, RB = L::RB, RC = L::RC, RT = L::RT, RU = L::RU;
  static constexpr int BF = eo_off(D1, Q, 0), GF = eo_off(D1, Q, 1), BT = eo_off(D1, Q, 2), GT = eo_off(D1, Q, 3);
  static constexpr int cD = (D1 + 1) / 2, hD = D1 / 2 > 0 ? D1 / 2 : 1;
  // phase A: X (region 0 until S1 ends), BB/GB/BG (region 0 from S2), BX/GX (region 1)
  __device__ static T* X(T* s) { return s; }
  __device__ static T* BX(T* s) { return s + L::R0; }
  __device__ static T* GX(T* s) { return s + L::R0 + Q * RB; }
  __device__ static T* BB(T* s) { return s; }
  __device__ static T* GB(T* s) { return s + Q * RC; }
  __device__ static T* BG(T* s) { return s + 2 * Q * RC; }
  // phase B
  __device__ static T* T0(T* s) { return s; }
  __device__ static T* T1(T* s) { return s + D1 * RT; }
  __device__ static T* T2(T* s) { return s + 2 * D1 * RT; }
  __device__ static T* UA(T* s) { return s + 3 * D1 * RT; }
  __device__ static T* UB(T* s) { return s + 3 * D1 * RT + D1 * RU; }

  // ---- diffusion
  // S1: line t = (z, y) along x -> BX, GX [qx][RB], column t
  __device__ static void d1(int t, T* s) {
    T xr[D1], e[cD], o[hD], bx[Q], gx[Q];
    const T* sx = X(s) + t * XP;
#pragma unroll
    for (int d = 0; d < D1; ++d) xr[d] = sx[d];
    eo_split<T, D1>(xr, e, o);
    eo_apply<T, Q, D1, 1, BF>(e, o, bx);
    eo_apply<T, Q, D1, -1, GF>(e, o, gx);
    T *sb = BX(s), *sg = GX(s);
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) {
      sb[qx * RB + t] = bx[qx];
      sg[qx * RB + t] = gx[qx];
    }
  }
  // S2: line t = (z, qx) along y -> BB, GB, BG [qy][RC], column t
  __device__ static void d2(int t, T* s) {
    const int z = t / Q, qx = t % Q;
    T br[D1], gr[D1], e[cD], o[hD], bb[Q], bg[Q], gb[Q];
    const T *sb = BX(s) + qx * RB + z * D1, *sg = GX(s) + qx * RB + z * D1;
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      br[d] = sb[d];
      gr[d] = sg[d];
    }
    eo_split<T, D1>(br, e, o);
    eo_apply<T, Q, D1, 1, BF>(e, o, bb);
    eo_apply<T, Q, D1, -1, GF>(e, o, bg);
    eo_line<T, Q, D1, 1, BF>(gr, gb);
    T *o0 = BB(s), *o1 = GB(s), *o2 = BG(s);
#pragma unroll
    for (int qy = 0; qy < Q; ++qy) {
      o0[qy * RC + t] = bb[qy];
      o1[qy * RC + t] = gb[qy];
      o2[qy * RC + t] = bg[qy];
    }
  }
  // S3: line t = (qy, qx) along z, D at every point, back along z; results
  // stay in registers until phase A is dead
  __device__ static void d3(int t, bool valid, const T* __restrict__ De, T* s, T* t0, T* t1, T* t2) {
    const int qy = t / Q, qx = t % Q;
    T rbb[D1], rgb[D1], rbg[D1], g0[Q], g1[Q], g2[Q];
    const T *sbb = BB(s) + qy * RC + qx, *sgb = GB(s) + qy * RC + qx, *sbg = BG(s) + qy * RC + qx;
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      rbb[z] = sbb[z * Q];
      rgb[z] = sgb[z * Q];
      rbg[z] = sbg[z * Q];
    }
    eo_line<T, Q, D1, 1, BF>(rgb, g0);
    eo_line<T, Q, D1, 1, BF>(rbg, g1);
    eo_line<T, Q, D1, -1, GF>(rbb, g2);
    const T* Dp = De + (size_t)t * 6;  // point-major: [q][6]
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) {
      T dd[6];
      if (valid) {
        d_load6(Dp + (size_t)qz * QQ * 6, dd);
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) dd[c] = 0;
      }
      const T d00 = dd[0], d01 = dd[1], d02 = dd[2], d11 = dd[3], d12 = dd[4], d22 = dd[5];
      const T a0 = g0[qz], a1 = g1[qz], a2 = g2[qz];
      g0[qz] = fe_norm(d00 * a0 + d01 * a1 + d02 * a2);
      g1[qz] = fe_norm(d01 * a0 + d11 * a1 + d12 * a2);
      g2[qz] = fe_norm(d02 * a0 + d12 * a1 + d22 * a2);
    }
    eo_line<T, D1, Q, 1, BT>(g0, t0);
    eo_line<T, D1, Q, 1, BT>(g1, t1);
    eo_line<T, D1, Q, -1, GT>(g2, t2);
  }
  __device__ static void d3_store(int t, T* s, const T* t0, const T* t1, const T* t2) {
    T *a = T0(s), *b = T1(s), *c = T2(s);
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      a[d * RT + t] = t0[d];
      b[d * RT + t] = t1[d];
      c[d * RT + t] = t2[d];
    }
  }
  // S4: line t = (dz, qx) along qy -> UA, UB [dy][RU], column t
  __device__ static void d4(int t, T* s) {
    const int dz = t / Q, qx = t % Q;
    T a0[Q], a1[Q], a2[Q], ua[D1], u1[D1], u2[D1];
    const T *s0 = T0(s) + dz * RT + qx, *s1 = T1(s) + dz * RT + qx, *s2 = T2(s) + dz * RT + qx;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      a0[q] = s0[q * Q];
      a1[q] = s1[q * Q];
      a2[q] = s2[q * Q];
    }
    eo_line<T, D1, Q, 1, BT>(a0, ua);
    eo_line<T, D1, Q, -1, GT>(a1, u1);
    eo_line<T, D1, Q, 1, BT>(a2, u2);
    T *oa = UA(s), *ob = UB(s);
#pragma unroll
    for (int dy = 0; dy < D1; ++dy) {
      oa[dy * RU + t] = ua[dy];
      ob[dy * RU + t] = fe_norm(u1[dy] + u2[dy]);
    }
  }
  // S5: line t = (dz, dy) along qx -> out[t * D1 + dx], or out[pos[t * D1 +
  // dx]] when pos (the element's DOF-sorted slot positions) is given
  template <typename TX>
  __device__ static void d5(int t, T* s, TX* __restrict__ out, const int32_t* __restrict__ pos = nullptr) {
    const int dz = t / D1, dy = t % D1;
    T ua[Q], ub[Q], y1[D1], y2[D1];
    const T *sa = UA(s) + dy * RU + dz * Q, *sb = UB(s) + dy * RU + dz * Q;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      ua[q] = sa[q];
      ub[q] = sb[q];
    }
    eo_line<T, D1, Q, -1, GT>(ua, y1);
    eo_line<T, D1, Q, 1, BT>(ub, y2);
    if (pos) {
#pragma unroll
      for (int dx = 0; dx < D1; ++dx) fe_store(&out[__ldg(pos + t * D1 + dx)], y1[dx] + y2[dx]);
    } else {
#pragma unroll
      for (int dx = 0; dx < D1; ++dx) fe_store(&out[t * D1 + dx], y1[dx] + y2[dx]);
    }
  }

  // ---- convection: the diffusion forward stages (d1, d2), then one value
  // per point v = D_q . gradhat (D_q = w adj(J) beta, point-major [q][3]),
  // then the mass backward stages (m3_store, m4, m5)
  __device__ static void c3(int t, bool valid, const T* __restrict__ De, T* s, T* t0) {
    const int qy = t / Q, qx = t % Q;
    T rbb[D1], rgb[D1], rbg[D1], g0[Q], g1[Q], g2[Q];
    const T *sbb = BB(s) + qy * RC + qx, *sgb = GB(s) + qy * RC + qx, *sbg = BG(s) + qy * RC + qx;
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      rbb[z] = sbb[z * Q];
      rgb[z] = sgb[z * Q];
      rbg[z] = sbg[z * Q];
    }
    eo_line<T, Q, D1, 1, BF>(rgb, g0);
    eo_line<T, Q, D1, 1, BF>(rbg, g1);
    eo_line<T, Q, D1, -1, GF>(rbb, g2);
    const T* Dp = De + (size_t)t * 3;
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) {
      T v = 0;
      if (valid) {
        const T* d = Dp + (size_t)qz * QQ * 3;
        v = fe_norm(fe_ldg(d) * g0[qz] + fe_ldg(d + 1) * g1[qz] + fe_ldg(d + 2) * g2[qz]);
      }
      g0[qz] = v;
    }
    eo_line<T, D1, Q, 1, BT>(g0, t0);
  }

  // ---- elasticity: three components, each with its own slab (component c
  // of the element at s + c * SE). The forward stages d1, d2 and the
  // backward stages d3_store, d4, d5 are the diffusion ones run on each
  // component; S3 couples the components through the stress at each point:
  //   H[c][r] = sum_s gh[c][s] M[s][r]          (physical gradient, M = J^-1)
  //   S = lw tr(H) I + mw (H + H^T)             (lw, mw = w det J lambda, mu)
  //   F[c][s] = sum_r S[c][r] M[s][r]           (= S J^-T)
  // out[c][0..2] are the back-z lines of F[c][0..2] (the t0, t1, t2 of d3).
  __device__ static void e3(int t, bool valid, const T* __restrict__ De, T* s, T (&out)[3][3][D1]) {
    const int qy = t / Q, qx = t % Q;
    T g[3][3][Q];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T* sc = s + c * L::SE3;
      T rbb[D1], rgb[D1], rbg[D1];
      const T *sbb = BB(sc) + qy * RC + qx, *sgb = GB(sc) + qy * RC + qx, *sbg = BG(sc) + qy * RC + qx;
#pragma unroll
      for (int z = 0; z < D1; ++z) {
        rbb[z] = sbb[z * Q];
        rgb[z] = sgb[z * Q];
        rbg[z] = sbg[z * Q];
      }
      eo_line<T, Q, D1, 1, BF>(rgb, g[c][0]);
      eo_line<T, Q, D1, 1, BF>(rbg, g[c][1]);
      eo_line<T, Q, D1, -1, GF>(rbb, g[c][2]);
    }
    const T* Dp = De + (size_t)t * 12;  // point-major: [q][12]
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) {
      T m[12];
      if (valid) {
        d_load12(Dp + (size_t)qz * QQ * 12, m);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) m[k] = 0;
      }
      T H[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          H[c][r] = fe_norm(g[c][0][qz] * m[r] + g[c][1][qz] * m[3 + r] + g[c][2][qz] * m[6 + r]);
      const T lt = fe_norm(m[9] * fe_norm(fe_norm(H[0][0] + H[1][1]) + H[2][2])), mw = m[10];
      T S[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) S[c][c] = fe_norm(lt + mw * fe_norm(H[c][c] + H[c][c]));
      S[0][1] = S[1][0] = fe_norm(mw * fe_norm(H[0][1] + H[1][0]));
      S[0][2] = S[2][0] = fe_norm(mw * fe_norm(H[0][2] + H[2][0]));
      S[1][2] = S[2][1] = fe_norm(mw * fe_norm(H[1][2] + H[2][1]));
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          g[c][a][qz] = fe_norm(S[c][0] * m[3 * a] + S[c][1] * m[3 * a + 1] + S[c][2] * m[3 * a + 2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      eo_line<T, D1, Q, 1, BT>(g[c][0], out[c][0]);
      eo_line<T, D1, Q, 1, BT>(g[c][1], out[c][1]);
      eo_line<T, D1, Q, -1, GT>(g[c][2], out[c][2]);
    }
  }

  // ---- mass (B only, one D per point)
  __device__ static void m1(int t, T* s) {
    T xr[D1], bx[Q];
    const T* sx = X(s) + t * XP;
#pragma unroll
    for (int d = 0; d < D1; ++d) xr[d] = sx[d];
    eo_line<T, Q, D1, 1, BF>(xr, bx);
    T* sb = BX(s);
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) sb[qx * RB + t] = bx[qx];
  }
  __device__ static void m2(int t, T* s) {
    const int z = t / Q, qx = t % Q;
    T br[D1], bb[Q];
    const T* sb = BX(s) + qx * RB + z * D1;
#pragma unroll
    for (int d = 0; d < D1; ++d) br[d] = sb[d];
    eo_line<T, Q, D1, 1, BF>(br, bb);
    T* o = BB(s);
#pragma unroll
    for (int qy = 0; qy < Q; ++qy) o[qy * RC + t] = bb[qy];
  }
  __device__ static void m3(int t, bool valid, const T* __restrict__ De, T* s, T* t0) {
    const int qy = t / Q, qx = t % Q;
    T rbb[D1], u[Q];
    const T* sbb = BB(s) + qy * RC + qx;
#pragma unroll
    for (int z = 0; z < D1; ++z) rbb[z] = sbb[z * Q];
    eo_line<T, Q, D1, 1, BF>(rbb, u);
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) u[qz] = valid ? fe_norm(fe_ldg(De + t + qz * QQ) * u[qz]) : T(0);
    eo_line<T, D1, Q, 1, BT>(u, t0);
  }
  __device__ static void m3_store(int t, T* s, const T* t0) {
    T* a = T0(s);
#pragma unroll
    for (int d = 0; d < D1; ++d) a[d * RT + t] = t0[d];
  }
  __device__ static void m4(int t, T* s) {
    const int dz = t / Q, qx = t % Q;
    T a0[Q], ua[D1];
    const T* s0 = T0(s) + dz * RT + qx;
#pragma unroll
    for (int q = 0; q < Q; ++q) a0[q] = s0[q * Q];
    eo_line<T, D1, Q, 1, BT>(a0, ua);
    T* oa = UA(s);
#pragma unroll
    for (int dy = 0; dy < D1; ++dy) oa[dy * RU + t] = ua[dy];
  }
  template <typename TX>
  __device__ static void m5(int t, T* s, TX* __restrict__ out, const int32_t* __restrict__ pos = nullptr) {
    const int dz = t / D1, dy = t % D1;
    T ua[Q], y[D1];
    const T* sa = UA(s) + dy * RU + dz * Q;
#pragma unroll
    for (int q = 0; q < Q; ++q) ua[q] = sa[q];
    eo_line<T, D1, Q, 1, BT>(ua, y);
    if (pos) {
#pragma unroll
      for (int dx = 0; dx < D1; ++dx) fe_store(&out[__ldg(pos + t * D1 + dx)], y[dx]);
    } else {
#pragma unroll
      for (int dx = 0; dx < D1; ++dx) fe_store(&out[t * D1 + dx], y[dx]);
    }
  }
};

#include "k_tc.cuh"

// ------------------------------------------------------------- drivers ----
// Thread tid's line in a stage of N lines per element with L lanes per
// element (ElemSmem::L1 / L2): element tid / L, line tid % L; lanes N .. L-1
// of an element and elements >= nel stay idle. L = N packs the lines of
// consecutive elements onto the lowest thread ids.
template <int N, int L>
__device__ __forceinline__ bool stage_line(int tid, int nel, int& el, int& t) {
  el = tid / L;
  t = tid - el * L;
  return el < nel && t < N;
}

// A block works on elements e0 .. e0 + nel - 1. The gather and stage S3
// (Q*Q lines per element) keep one plane of Q*Q threads per element, thread
// tid = el * Q*Q + t (threads of planes el >= nel take part with valid =
// false; the block needs a slab for every plane it has); the stages with
// fewer lines (S1, S5: D1^2; S2, S4: D1*Q) either pack the lines of the
// nel elements onto the lowest thread ids, so warps are full and the
// arithmetic pipe issues no instructions for idle lanes (FP64, double-float),
// or give each element whole warps (FP32 where the plane has the lanes;
// stage_lanes). Element e's DOF list is
// e2l + e*D1^3, its D block Dq + e*NC*Q^3 (NC = 6 diffusion, 1 mass), its
// E-vector slice ye + e*D1^3 (or, with pos, the positions pos[e*D1^3 + k]
// of the DOF-sorted E-vector ye); its slab sm + el*SE. Every thread of the
// block must call the driver (it contains __syncthreads).
template <typename T, int D1, int Q, typename TX = T>
__device__ __forceinline__ void diffusion_block(int tid, int e0, int nel, const int32_t* __restrict__ e2l,
                                                const T* __restrict__ Dq, T* sm, const TX* __restrict__ x,
                                                TX* __restrict__ ye, const int32_t* __restrict__ pos = nullptr) {
  using Ln = Lines<T, D1, Q>;
  constexpr int QQ = Q * Q, ND = D1 * D1 * D1, NQ = Q * Q * Q, SE = ElemSmem<T, D1, Q>::SE;
  constexpr int N1 = D1 * D1, N2 = D1 * Q, L1 = ElemSmem<T, D1, Q>::L1, L2 = ElemSmem<T, D1, Q>::L2;
  const int el = tid / QQ, t = tid % QQ;
  const bool valid = el < nel;
  const size_t ev = valid ? (size_t)(e0 + el) : 0;
  int se, st;  // element and line of the short stages
  gather_x<T, D1, Q, TX>(t, valid, e2l + ev * ND, x, Ln::X(sm + el * SE), Ln::XP);
  __syncthreads();
  if constexpr (use_tc<T, D1>()) {
    tc_s1<D1, Q>(nel * N1, sm, tid, blockDim.x * blockDim.y * blockDim.z);
  } else {
    if (stage_line<N1, L1>(tid, nel, se, st)) Ln::d1(st, sm + se * SE);
  }
  __syncthreads();
  if (stage_line<N2, L2>(tid, nel, se, st)) Ln::d2(st, sm + se * SE);
  __syncthreads();
  T t0[D1], t1[D1], t2[D1];
  Ln::d3(t, valid, Dq + ev * 6 * NQ, sm + el * SE, t0, t1, t2);
  __syncthreads();
  Ln::d3_store(t, sm + el * SE, t0, t1, t2);
  __syncthreads();
  if (stage_line<N2, L2>(tid, nel, se, st)) Ln::d4(st, sm + se * SE);
  __syncthreads();
  if constexpr (use_tc<T, D1>()) {
    tc_s5<D1, Q, TX>(nel * N1, sm, tid, blockDim.x * blockDim.y * blockDim.z, ye + (pos ? 0 : (size_t)e0 * ND),
                     pos ? pos + (size_t)e0 * ND : nullptr);
  } else if (stage_line<N1, L1>(tid, nel, se, st)) {
    const size_t eo = (size_t)(e0 + se) * ND;
    if (pos) Ln::template d5<TX>(st, sm + se * SE, ye, pos + eo);
    else Ln::template d5<TX>(st, sm + se * SE, ye + eo);
  }
}

// Convection (beta . grad u, v): forward stages of diffusion, backward
// stages of mass; D block Dq + e*3*Q^3.
template <typename T, int D1, int Q, typename TX = T>
__device__ __forceinline__ void convection_block(int tid, int e0, int nel, const int32_t* __restrict__ e2l,
                                                 const T* __restrict__ Dq, T* sm, const TX* __restrict__ x,
                                                 TX* __restrict__ ye, const int32_t* __restrict__ pos = nullptr) {
  using Ln = Lines<T, D1, Q>;
  constexpr int QQ = Q * Q, ND = D1 * D1 * D1, NQ = Q * Q * Q, SE = ElemSmem<T, D1, Q>::SE;
  constexpr int N1 = D1 * D1, N2 = D1 * Q, L1 = ElemSmem<T, D1, Q>::L1, L2 = ElemSmem<T, D1, Q>::L2;
  const int el = tid / QQ, t = tid % QQ;
  const bool valid = el < nel;
  const size_t ev = valid ? (size_t)(e0 + el) : 0;
  int se, st;
  gather_x<T, D1, Q, TX>(t, valid, e2l + ev * ND, x, Ln::X(sm + el * SE), Ln::XP);
  __syncthreads();
  if (stage_line<N1, L1>(tid, nel, se, st)) Ln::d1(st, sm + se * SE);
  __syncthreads();
  if (stage_line<N2, L2>(tid, nel, se, st)) Ln::d2(st, sm + se * SE);
  __syncthreads();
  T t0[D1];
  Ln::c3(t, valid, Dq + ev * 3 * NQ, sm + el * SE, t0);
  __syncthreads();
  Ln::m3_store(t, sm + el * SE, t0);
  __syncthreads();
  if (stage_line<N2, L2>(tid, nel, se, st)) Ln::m4(st, sm + se * SE);
  __syncthreads();
  if (stage_line<N1, L1>(tid, nel, se, st)) {
    const size_t eo = (size_t)(e0 + se) * ND;
    if (pos) Ln::template m5<TX>(st, sm + se * SE, ye, pos + eo);
    else Ln::template m5<TX>(st, sm + se * SE, ye + eo);
  }
}

template <typename T, int D1, int Q, typename TX = T>
__device__ __forceinline__ void mass_block(int tid, int e0, int nel, const int32_t* __restrict__ e2l,
                                           const T* __restrict__ Dq, T* sm, const TX* __restrict__ x,
                                           TX* __restrict__ ye, const int32_t* __restrict__ pos = nullptr) {
  using Ln = Lines<T, D1, Q>;
  constexpr int QQ = Q * Q, ND = D1 * D1 * D1, NQ = Q * Q * Q, SE = ElemSmem<T, D1, Q>::SE;
  constexpr int N1 = D1 * D1, N2 = D1 * Q, L1 = ElemSmem<T, D1, Q>::L1, L2 = ElemSmem<T, D1, Q>::L2;
  const int el = tid / QQ, t = tid % QQ;
  const bool valid = el < nel;
  const size_t ev = valid ? (size_t)(e0 + el) : 0;
  int se, st;
  gather_x<T, D1, Q, TX>(t, valid, e2l + ev * ND, x, Ln::X(sm + el * SE), Ln::XP);
  __syncthreads();
  if (stage_line<N1, L1>(tid, nel, se, st)) Ln::m1(st, sm + se * SE);
  __syncthreads();
  if (stage_line<N2, L2>(tid, nel, se, st)) Ln::m2(st, sm + se * SE);
  __syncthreads();
  T t0[D1];
  Ln::m3(t, valid, Dq + ev * NQ, sm + el * SE, t0);
  __syncthreads();
  Ln::m3_store(t, sm + el * SE, t0);
  __syncthreads();
  if (stage_line<N2, L2>(tid, nel, se, st)) Ln::m4(st, sm + se * SE);
  __syncthreads();
  if (stage_line<N1, L1>(tid, nel, se, st)) {
    const size_t eo = (size_t)(e0 + se) * ND;
    if (pos) Ln::template m5<TX>(st, sm + se * SE, ye, pos + eo);
    else Ln::template m5<TX>(st, sm + se * SE, ye + eo);
  }
}

// Linear elasticity on the three components of a vector H1 field
// (component-major vectors: component c of DOF i at c * ndof + i; E-vector
// [3][ne][D1^3]). The block's NT threads own NE planes of Q*Q threads for
// S3 (one point line of one element each); every other stage loops its
// lines of all (element, component) slabs over the block's threads, slab
// (el, c) at sm + (3 el + c) SE. D block: Dq + e * 12 Q^3.
template <typename T, int D1, int Q, int NT, typename TX = T>
__device__ __forceinline__ void elasticity_block(int tid, int e0, int nel, int ne, int64_t ndof,
                                                 const int32_t* __restrict__ e2l, const T* __restrict__ Dq, T* sm,
                                                 const TX* __restrict__ x, TX* __restrict__ ye,
                                                 const int32_t* __restrict__ pos = nullptr) {
  using Ln = Lines<T, D1, Q>;
  constexpr int QQ = Q * Q, ND = D1 * D1 * D1, NQ = Q * Q * Q, SE = ElemSmem<T, D1, Q>::SE3;
  constexpr int N1 = D1 * D1, N2 = D1 * Q, XP = Ln::XP;
  // gather: one map entry, three component values
  for (int i = tid; i < nel * ND; i += NT) {
    const int el = i / ND, k = i % ND;
    const int32_t g = __ldg(e2l + (size_t)(e0 + el) * ND + k);
    const TX v0 = __ldg(x + g), v1 = __ldg(x + ndof + g), v2 = __ldg(x + 2 * ndof + g);
    T* sx = sm + 3 * el * SE + (k / D1) * XP + k % D1;
    sx[0] = fe_from<T>(v0);
    sx[SE] = fe_from<T>(v1);
    sx[2 * SE] = fe_from<T>(v2);
  }
  __syncthreads();
  for (int i = tid; i < 3 * nel * N1; i += NT) Ln::d1(i % N1, sm + (i / N1) * SE);
  __syncthreads();
  for (int i = tid; i < 3 * nel * N2; i += NT) Ln::d2(i % N2, sm + (i / N2) * SE);
  __syncthreads();
  const int el = tid / QQ, t = tid % QQ;
  const bool valid = el < nel;
  const size_t ev = valid ? (size_t)(e0 + el) : 0;
  T out[3][3][D1];
  Ln::e3(t, valid, Dq + ev * 12 * NQ, sm + 3 * el * SE, out);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) Ln::d3_store(t, sm + (3 * el + c) * SE, out[c][0], out[c][1], out[c][2]);
  __syncthreads();
  for (int i = tid; i < 3 * nel * N2; i += NT) Ln::d4(i % N2, sm + (i / N2) * SE);
  __syncthreads();
  for (int i = tid; i < 3 * nel * N1; i += NT) {
    const int sl = i / N1, l = sl / 3, c = sl % 3;
    if (pos)  // component c's DOF-sorted E-vector at ye + c ne ND
      Ln::template d5<TX>(i % N1, sm + sl * SE, ye + (size_t)c * ne * ND, pos + (size_t)(e0 + l) * ND);
    else
      Ln::template d5<TX>(i % N1, sm + sl * SE, ye + ((size_t)c * ne + e0 + l) * ND);
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
