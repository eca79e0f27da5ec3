// 1D basis tables of every compiled (p, q) pair in constant memory.
//
// B1d[k][j] = l_j(x_k) and G1d[k][j] = l_j'(x_k) depend only on (p, q) (GLL
// nodes, Gauss points), so the element kernels read them from constant memory
// at indices that are compile-time constants once the contraction loops are
// unrolled: each coefficient becomes an operand of the FMA instruction itself
// and costs no load. Constant memory is per translation unit (no relocatable
// device code), so every .cu file that includes this header fills its own copy
// through fem_tables_ensure(), once per device, from the host tables of
// fem_basis.cpp. Call it from a set-up entry point, never inside a stream
// capture (it copies to the device synchronously).
#pragma once

#include <mutex>
#include <vector>

#include "fem_internal.h"
#include "k_df64.cuh"

// (D1, Q) pairs in the order of FEM_FOR_EACH_PQ; entries D1 * Q each.
__host__ __device__ constexpr int tab_off(int D1, int Q) {
  const int pairs[16][2] = {{2, 2}, {2, 3}, {3, 3}, {3, 4}, {4, 4}, {4, 5}, {5, 5}, {5, 6},
                            {6, 6}, {6, 7}, {7, 7}, {7, 8}, {8, 8}, {8, 9}, {9, 9}, {9, 10}};
  int off = 0;
  for (int i = 0; i < 16; ++i) {
    if (pairs[i][0] == D1 && pairs[i][1] == Q) return off;
    off += pairs[i][0] * pairs[i][1];
  }
  return -1;
}
constexpr int kTabTotal = tab_off(9, 10) + 90;

static __constant__ double c_B64[kTabTotal];
static __constant__ double c_G64[kTabTotal];
static __constant__ float c_B32[kTabTotal];
static __constant__ float c_G32[kTabTotal];
static __constant__ float c_Bhi[kTabTotal];
static __constant__ float c_Blo[kTabTotal];
static __constant__ float c_Ghi[kTabTotal];
static __constant__ float c_Glo[kTabTotal];

// Even-odd ("folded") forms of the 1D operators. GLL nodes and Gauss points
// are symmetric about 1/2, so B[Q-1-k][D1-1-j] = B[k][j] and
// G[Q-1-k][D1-1-j] = -G[k][j]; the same holds for the transposes. For a
// matrix A (M x K) with A[M-1-k][K-1-j] = s A[k][j] and a line x, write
// e_j = x_j + x_{K-1-j}, o_j = x_j - x_{K-1-j} (j < K/2), e_{K/2} = x_mid:
//   P_k = sum_j AP[k][j] e_j,  N_k = sum_j AN[k][j] o_j,
//   y_k = P_k + N_k,  y_{M-1-k} = s (P_k - N_k)   (k < M/2),
// AP[k][j] = (A[k][j] + A[k][K-1-j]) / 2, AP[k][K/2] = A[k][mid],
// AN[k][j] = (A[k][j] - A[k][K-1-j]) / 2, and a middle output (M odd) is P
// (s = 1) or N (s = -1). Tables per (D1, Q): forward B, G (M = Q, K = D1)
// and transposed B, G (M = D1, K = Q), each as AP [ceil(M/2)][ceil(K/2)]
// followed by AN [ceil(M/2)][K/2].
__host__ __device__ constexpr int eo_size(int M, int K) { return ((M + 1) / 2) * K; }
__host__ __device__ constexpr int eo_pair_size(int D1, int Q) { return 2 * eo_size(Q, D1) + 2 * eo_size(D1, Q); }
// which: 0 B forward, 1 G forward, 2 B transposed, 3 G transposed
__host__ __device__ constexpr int eo_off(int D1, int Q, int which) {
  const int pairs[16][2] = {{2, 2}, {2, 3}, {3, 3}, {3, 4}, {4, 4}, {4, 5}, {5, 5}, {5, 6},
                            {6, 6}, {6, 7}, {7, 7}, {7, 8}, {8, 8}, {8, 9}, {9, 9}, {9, 10}};
  int off = 0;
  for (int i = 0; i < 16; ++i) {
    if (pairs[i][0] == D1 && pairs[i][1] == Q) {
      const int f = eo_size(Q, D1), t = eo_size(D1, Q);
      return off + (which == 0 ? 0 : which == 1 ? f : which == 2 ? 2 * f : 2 * f + t);
    }
    off += eo_pair_size(pairs[i][0], pairs[i][1]);
  }
  return -1;
}
constexpr int kEOTotal = eo_off(9, 10, 0) + eo_pair_size(9, 10);

static __constant__ double c_EO64[kEOTotal];
static __constant__ float c_EO32[kEOTotal];
static __constant__ float c_EOhi[kEOTotal];
static __constant__ float c_EOlo[kEOTotal];

template <typename T>
struct EO;
template <>
struct EO<double> {
  __device__ __forceinline__ static double c(int i) { return c_EO64[i]; }
};
template <>
struct EO<float> {
  __device__ __forceinline__ static float c(int i) { return c_EO32[i]; }
};
template <>
struct EO<df64> {
  __device__ __forceinline__ static df64 c(int i) { return df64(c_EOhi[i], c_EOlo[i]); }
};

// Host: folded table of the M x K matrix A (row-major) into out.
static void eo_fold(const std::vector<double>& A, int M, int K, double* out) {
  const int cM = (M + 1) / 2, cK = (K + 1) / 2, hK = K / 2;
  for (int k = 0; k < cM; ++k) {
    for (int j = 0; j < hK; ++j) out[k * cK + j] = 0.5 * (A[k * K + j] + A[k * K + K - 1 - j]);
    if (K & 1) out[k * cK + hK] = A[k * K + hK];
    for (int j = 0; j < hK; ++j) out[cM * cK + k * hK + j] = 0.5 * (A[k * K + j] - A[k * K + K - 1 - j]);
  }
}

template <typename T>
struct Tab;
template <>
struct Tab<double> {
  __device__ __forceinline__ static double B(int i) { return c_B64[i]; }
  __device__ __forceinline__ static double G(int i) { return c_G64[i]; }
};
template <>
struct Tab<float> {
  __device__ __forceinline__ static float B(int i) { return c_B32[i]; }
  __device__ __forceinline__ static float G(int i) { return c_G32[i]; }
};
template <>
struct Tab<df64> {
  __device__ __forceinline__ static df64 B(int i) { return df64(c_Bhi[i], c_Blo[i]); }
  __device__ __forceinline__ static df64 G(int i) { return df64(c_Ghi[i], c_Glo[i]); }
};

// Fill this translation unit's tables on the current device (once).
static fem_status fem_tables_ensure() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  FEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fem_fail(FEM_EUNSUPPORTED, "tables: device index %d", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return FEM_OK;
  std::vector<double> b64(kTabTotal), g64(kTabTotal);
  const int pairs[16][2] = {{2, 2}, {2, 3}, {3, 3}, {3, 4}, {4, 4}, {4, 5}, {5, 5}, {5, 6},
                            {6, 6}, {6, 7}, {7, 7}, {7, 8}, {8, 8}, {8, 9}, {9, 9}, {9, 10}};
  for (int i = 0; i < 16; ++i) {
    const int D1 = pairs[i][0], Q = pairs[i][1];
    std::vector<double> nodes, pts, wts, B, G;
    fem_gll_nodes(D1 - 1, nodes);
    fem_gauss_rule(Q, pts, wts);
    fem_lagrange_tables(nodes, pts, B, G);
    const int off = tab_off(D1, Q);
    for (int k = 0; k < D1 * Q; ++k) {
      b64[off + k] = B[k];
      g64[off + k] = G[k];
    }
  }
  // folded tables
  std::vector<double> eo(kEOTotal, 0.0);
  for (int i = 0; i < 16; ++i) {
    const int D1 = pairs[i][0], Q = pairs[i][1], off = tab_off(D1, Q);
    std::vector<double> Bf(b64.begin() + off, b64.begin() + off + D1 * Q), Gf(g64.begin() + off, g64.begin() + off + D1 * Q);
    std::vector<double> Bt(D1 * Q), Gt(D1 * Q);  // transposes: [D1][Q]
    for (int k = 0; k < Q; ++k)
      for (int j = 0; j < D1; ++j) {
        Bt[j * Q + k] = Bf[k * D1 + j];
        Gt[j * Q + k] = Gf[k * D1 + j];
      }
    eo_fold(Bf, Q, D1, eo.data() + eo_off(D1, Q, 0));
    eo_fold(Gf, Q, D1, eo.data() + eo_off(D1, Q, 1));
    eo_fold(Bt, D1, Q, eo.data() + eo_off(D1, Q, 2));
    eo_fold(Gt, D1, Q, eo.data() + eo_off(D1, Q, 3));
  }
  std::vector<float> eo32(kEOTotal), eohi(kEOTotal), eolo(kEOTotal);
  for (int k = 0; k < kEOTotal; ++k) {
    eo32[k] = (float)eo[k];
    eohi[k] = (float)eo[k];
    eolo[k] = (float)(eo[k] - (double)eohi[k]);
  }
  FEM_CUDA(cudaMemcpyToSymbol(c_EO64, eo.data(), sizeof(double) * kEOTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_EO32, eo32.data(), sizeof(float) * kEOTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_EOhi, eohi.data(), sizeof(float) * kEOTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_EOlo, eolo.data(), sizeof(float) * kEOTotal));
  std::vector<float> b32(kTabTotal), g32(kTabTotal), bhi(kTabTotal), blo(kTabTotal), ghi(kTabTotal),
      glo(kTabTotal);
  for (int k = 0; k < kTabTotal; ++k) {
    b32[k] = (float)b64[k];
    g32[k] = (float)g64[k];
    bhi[k] = (float)b64[k];
    blo[k] = (float)(b64[k] - (double)bhi[k]);
    ghi[k] = (float)g64[k];
    glo[k] = (float)(g64[k] - (double)ghi[k]);
  }
  FEM_CUDA(cudaMemcpyToSymbol(c_B64, b64.data(), sizeof(double) * kTabTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_G64, g64.data(), sizeof(double) * kTabTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_B32, b32.data(), sizeof(float) * kTabTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_G32, g32.data(), sizeof(float) * kTabTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_Bhi, bhi.data(), sizeof(float) * kTabTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_Blo, blo.data(), sizeof(float) * kTabTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_Ghi, ghi.data(), sizeof(float) * kTabTotal));
  FEM_CUDA(cudaMemcpyToSymbol(c_Glo, glo.data(), sizeof(float) * kTabTotal));
  done[dev] = true;
  return FEM_OK;
}
