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
