// Device helpers shared by the library's CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fem_internal.h"

// Grid for a grid-stride loop over `total` items: at most 8 resident blocks of
// `threads` threads on each of the device's SMs (152 on GB300).
int fem_sm_count();
inline int grid_for(int64_t total, int threads) {
  if (total <= 0) return 1;
  const int64_t need = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)fem_sm_count() * 8;
  return (int)(need < cap ? need : cap);
}

// Deterministic block sum of one double per thread (fixed shuffle tree, then
// warp partials in smem summed by warp 0 in a fixed order). Result valid in
// thread 0. `red` needs blockDim.x / 32 doubles. All threads must call it.
__device__ inline double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += red[w];
  }
  return s;
}

// Per-thread accumulator of a dot product over vectors of type T. A thread
// sums a few tens of terms before the FP64 block and grid sums; FP32 vectors
// accumulate those terms in FP32 on the FP32 pipe (converting every term to
// FP64 put two conversions and a DFMA per term on the FP64 pipe, which then
// bound the FP32 solver's vector kernels), FP64 vectors in FP64.
template <typename T>
struct DotAcc {
  using type = double;
};
template <>
struct DotAcc<float> {
  using type = float;
};

// Compiled (p, q1d) set: q1d = p + 2 (the Gauss rule of the benchmark
// workloads) and q1d = p + 1, for p = 1..8.
#define FEM_FOR_EACH_PQ(X) \
  X(1, 2) X(1, 3) X(2, 3) X(2, 4) X(3, 4) X(3, 5) X(4, 5) X(4, 6) \
  X(5, 6) X(5, 7) X(6, 7) X(6, 8) X(7, 8) X(7, 9) X(8, 9) X(8, 10)

// Orders compiled into the persistent batched kernel (one kernel holds every
// variant, so its register count is the maximum over them): p = 1..6.
#define FEM_FOR_EACH_PQ_BATCH(X) \
  X(1, 2) X(1, 3) X(2, 3) X(2, 4) X(3, 4) X(3, 5) X(4, 5) X(4, 6) X(5, 6) X(5, 7) X(6, 7) X(6, 8)
