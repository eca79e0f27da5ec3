// Tensor-core form of the x-direction stages of the FP32 diffusion element
// operator (build option FEM_F32_TC=1; the line form of k_element.cuh
// otherwise). S1 and S5 are small dense products over the block's lines:
//   S1: [lines (el, z, y)] x [x = 0..D1-1]  times  W1[x][n] = (B | G)[n][x]
//   S5: [lines (el, dz, dy)] x [k = qx of UA | qx of UB]  times
//       W5[k][dx] = (G | B)[qx][dx]
// Each warp takes 16 lines at a time and runs mma.sync m16n8k8 with TF32
// operands and FP32 accumulation, in the split form (a = a_hi + a_lo,
// w = w_hi + w_lo, a w ~ a_lo w_hi + a_hi w_lo + a_hi w_hi with every part
// TF32) that keeps FP32-level accuracy. Zero padding fills K and N up to
// multiples of 8. Fragment layouts (PTX ISA, mma.m16n8k8 .tf32): with
// g = lane / 4 and c = lane % 4, A holds (g, c), (g + 8, c), (g, c + 4),
// (g + 8, c + 4); B holds (k = c, n = g), (k = c + 4, n = g); the
// accumulator (g, 2c), (g, 2c + 1), (g + 8, 2c), (g + 8, 2c + 1).
#pragma once

#include <stdint.h>

#include "k_tables.cuh"

#ifndef FEM_F32_TC
#define FEM_F32_TC 0
#endif

// Whether the FP32 element kernel of order D1 - 1 uses the tensor-core S1/S5.
template <typename T, int D1>
constexpr bool use_tc() {
  return FEM_F32_TC != 0 && std::is_same<T, float>::value && D1 >= 5;
}

__device__ __forceinline__ uint32_t tf32_of(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// v = hi + lo with both parts TF32.
__device__ __forceinline__ void tf32_split(float v, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(v);
  lo = tf32_of(v - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += a w in split TF32 (three products, small terms first); FEM_F32_TC=2
// takes the single TF32 product instead (about 1e-3 relative error).
__device__ __forceinline__ void mma3(float (&d)[4], const float (&a)[4], float w0, float w1) {
  if (FEM_F32_TC == 2) {
    uint32_t ah[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) ah[i] = tf32_of(a[i]);
    mma_tf32(d, ah, tf32_of(w0), tf32_of(w1));
    return;
  }
  uint32_t ah[4], al[4], wh0, wl0, wh1, wl1;
#pragma unroll
  for (int i = 0; i < 4; ++i) tf32_split(a[i], ah[i], al[i]);
  tf32_split(w0, wh0, wl0);
  tf32_split(w1, wh1, wl1);
  mma_tf32(d, al, wh0, wh1);
  mma_tf32(d, ah, wl0, wl1);
  mma_tf32(d, ah, wh0, wh1);
}

// S1 over nlines = nel * D1^2 lines (line L: element L / D1^2, line L % D1^2
// of its slab). Called by every thread of the block (no barrier inside).
template <int D1, int Q>
__device__ __forceinline__ void tc_s1(int nlines, float* sm, int tid, int nthreads) {
  using L = ElemSmem<float, D1, Q>;
  constexpr int N1 = D1 * D1, SE = L::SE, XP = L::XP, RB = L::RB, R0 = L::R0;
  constexpr int KS = (D1 + 7) / 8, NT = (2 * Q + 7) / 8, OFF = tab_off(D1, Q);
  // mma.sync needs all 32 lanes: a partial last warp (Q^2 NE not a multiple
  // of 32) takes no tiles
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
  if (warp >= nwarps) return;
  const int g = lane >> 2, c = lane & 3;
  for (int tile = warp; tile * 16 < nlines; tile += nwarps) {
    const int L0 = tile * 16 + g, L1 = L0 + 8;
    const bool v0 = L0 < nlines, v1 = L1 < nlines;
    const float* x0 = v0 ? sm + (L0 / N1) * SE + (L0 % N1) * XP : sm;
    const float* x1 = v1 ? sm + (L1 / N1) * SE + (L1 % N1) * XP : sm;
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[nt][i] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const int k0 = ks * 8 + c, k1 = k0 + 4;
      float a[4];
      a[0] = (v0 && k0 < D1) ? x0[k0] : 0.0f;
      a[1] = (v1 && k0 < D1) ? x1[k0] : 0.0f;
      a[2] = (v0 && k1 < D1) ? x0[k1] : 0.0f;
      a[3] = (v1 && k1 < D1) ? x1[k1] : 0.0f;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int n = nt * 8 + g;
        // W1[k][n] = B[n][k] (n < Q), G[n - Q][k] (Q <= n < 2Q)
        float w0 = 0.0f, w1 = 0.0f;
        if (n < Q) {
          if (k0 < D1) w0 = Tab<float>::B(OFF + n * D1 + k0);
          if (k1 < D1) w1 = Tab<float>::B(OFF + n * D1 + k1);
        } else if (n < 2 * Q) {
          if (k0 < D1) w0 = Tab<float>::G(OFF + (n - Q) * D1 + k0);
          if (k1 < D1) w1 = Tab<float>::G(OFF + (n - Q) * D1 + k1);
        }
        mma3(acc[nt], a, w0, w1);
      }
    }
    // BX / GX [qx][RB] at column = line within the element
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int n = nt * 8 + 2 * c + h;
        if (n >= 2 * Q) continue;
        float* base0 = v0 ? sm + (L0 / N1) * SE + R0 : nullptr;
        float* base1 = v1 ? sm + (L1 / N1) * SE + R0 : nullptr;
        const int col = n < Q ? n * RB : Q * RB + (n - Q) * RB;
        if (v0) base0[col + L0 % N1] = acc[nt][h];
        if (v1) base1[col + L1 % N1] = acc[nt][2 + h];
      }
    }
  }
}

// S5 over nlines = nel * D1^2 lines (line L: element L / D1^2, t = L % D1^2 =
// (dz, dy)); output out[el * D1^3 + t * D1 + dx] (with pos: at out[pos[...]]).
template <int D1, int Q, typename TX>
__device__ __forceinline__ void tc_s5(int nlines, float* sm, int tid, int nthreads, TX* __restrict__ out,
                                      const int32_t* __restrict__ pos = nullptr) {
  using L = ElemSmem<float, D1, Q>;
  constexpr int N1 = D1 * D1, ND = D1 * D1 * D1, SE = L::SE, RU = L::RU, RT = L::RT;
  constexpr int KS = (2 * Q + 7) / 8, NT = (D1 + 7) / 8, OFF = tab_off(D1, Q);
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;  // full warps only
  if (warp >= nwarps) return;
  const int g = lane >> 2, c = lane & 3;
  for (int tile = warp; tile * 16 < nlines; tile += nwarps) {
    const int L0 = tile * 16 + g, L1 = L0 + 8;
    const bool v0 = L0 < nlines, v1 = L1 < nlines;
    // UA at slab + 3 D1 RT, UB at UA + D1 RU; row (dz, dy) reads [dy][RU] + dz Q + qx
    const float* u0 = sm;
    const float* u1 = sm;
    if (v0) {
      const int t = L0 % N1;
      u0 = sm + (L0 / N1) * SE + 3 * D1 * RT + (t % D1) * RU + (t / D1) * Q;
    }
    if (v1) {
      const int t = L1 % N1;
      u1 = sm + (L1 / N1) * SE + 3 * D1 * RT + (t % D1) * RU + (t / D1) * Q;
    }
    float acc[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[nt][i] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const int k0 = ks * 8 + c, k1 = k0 + 4;
      // k < Q: UA[qx = k]; Q <= k < 2Q: UB[qx = k - Q] (UB = UA + D1 RU)
      auto ld = [&](const float* u, bool v, int k) -> float {
        if (!v || k >= 2 * Q) return 0.0f;
        return k < Q ? u[k] : u[D1 * RU + (k - Q)];
      };
      float a[4] = {ld(u0, v0, k0), ld(u1, v1, k0), ld(u0, v0, k1), ld(u1, v1, k1)};
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int n = nt * 8 + g;  // dx
        // W5[k][dx] = G[k][dx] (k < Q), B[k - Q][dx] (Q <= k < 2Q)
        auto w = [&](int k) -> float {
          if (n >= D1 || k >= 2 * Q) return 0.0f;
          return k < Q ? Tab<float>::G(OFF + k * D1 + n) : Tab<float>::B(OFF + (k - Q) * D1 + n);
        };
        mma3(acc[nt], a, w(k0), w(k1));
      }
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int dx = nt * 8 + 2 * c + h;
        if (dx >= D1) continue;
        const size_t i0 = (size_t)(L0 / N1) * ND + (L0 % N1) * D1 + dx;
        const size_t i1 = (size_t)(L1 / N1) * ND + (L1 % N1) * D1 + dx;
        if (v0) fe_store(&out[pos ? (size_t)__ldg(pos + i0) : i0], acc[nt][h]);
        if (v1) fe_store(&out[pos ? (size_t)__ldg(pos + i1) : i1], acc[nt][2 + h]);
      }
    }
  }
}
