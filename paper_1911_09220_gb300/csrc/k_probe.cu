// Arithmetic-peak probe: the FP64 and FP32 fused multiply-add rates of the
// device this library runs on, measured with CUDA events around one kernel
// that keeps eight independent FMA chains per thread in flight on every SM
// (best of three launches after a warm-up launch of the same length).
// The paper has no counterpart: these rates are the denominators of the
// roofline fractions that the element kernels, bound by their arithmetic
// pipes (FP64 DFMA on GB300 is 1/64 of the FP32 rate), are quoted against.
#include "fem_internal.h"
#include "k_common.cuh"

namespace {

__device__ double g_probe_sink64;
__device__ float g_probe_sink32;

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

// Each thread runs kChains independent chains a = a * b + c for `iters`
// steps (2 flops per step and chain); the sum of the chains is written only
// if it equals a value it cannot reach, so the work stays live without
// memory traffic.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T b, T c, T* sink) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = a[k] * b + c;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == (T)-1.2345e30) *sink = s;
}

template <typename T>
fem_status run_probe(T* sink, int iters, cudaStream_t s, double* tflops) {
  int blocks_per_sm = 0;
  FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_fma_probe<T>, kProbeThreads, 0));
  const int grid = fem_sm_count() * (blocks_per_sm > 0 ? blocks_per_sm : 1);
  // b slightly below 1 and c small keep every chain finite and normal
  const T b = (T)0.999999, c = (T)1e-6;
  // warm-up (lets the clocks ramp), then the best of three timed launches
  k_fma_probe<T><<<grid, kProbeThreads, 0, s>>>(iters, b, c, sink);
  FEM_LAUNCHED();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FEM_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fem_fail(FEM_ECUDA, "fem_probe_fma_peak: cudaEventCreate failed");
  }
  float best = 0.0f;
  bool ok = true;
  for (int rep = 0; rep < 3 && ok; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_probe<T><<<grid, kProbeThreads, 0, s>>>(iters, b, c, sink);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
         cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f;
    if (ok && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return fem_fail(FEM_ECUDA, "fem_probe_fma_peak: probe launch or timing failed");
  const double flops = 2.0 * kChains * (double)iters * grid * kProbeThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return FEM_OK;
}

}  // namespace

extern "C" fem_status fem_probe_fma_peak(int dtype, int iters, double* tflops, void* stream) {
  if (!tflops || iters <= 0) return fem_fail(FEM_EINVAL, "fem_probe_fma_peak: tflops != NULL and iters > 0 required");
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == FEM_F64) {
    double* sink = nullptr;
    FEM_CUDA(cudaGetSymbolAddress((void**)&sink, g_probe_sink64));
    return run_probe<double>(sink, iters, s, tflops);
  }
  if (dtype == FEM_F32) {
    float* sink = nullptr;
    FEM_CUDA(cudaGetSymbolAddress((void**)&sink, g_probe_sink32));
    return run_probe<float>(sink, iters, s, tflops);
  }
  return fem_fail(FEM_EINVAL, "fem_probe_fma_peak: dtype must be FEM_F64 or FEM_F32");
}
