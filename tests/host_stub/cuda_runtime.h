/*
 * Test-only stand-in for the CUDA runtime header, used to compile the
 * library's host sources (fem_host.cpp, fem_basis.cpp) into a CPU-only test
 * library: "device" memory is host memory and copies are memcpy. Declares
 * only what those sources use. Never part of the product build.
 */
#pragma once
#include <stddef.h>

typedef enum { cudaSuccess = 0, cudaErrorMemoryAllocation = 2, cudaErrorInvalidValue = 1 } cudaError_t;
typedef enum {
  cudaMemcpyHostToHost = 0,
  cudaMemcpyHostToDevice = 1,
  cudaMemcpyDeviceToHost = 2,
  cudaMemcpyDeviceToDevice = 3,
  cudaMemcpyDefault = 4
} cudaMemcpyKind;
typedef struct CUstream_st* cudaStream_t;

cudaError_t cudaMalloc(void** p, size_t bytes);
cudaError_t cudaFree(void* p);
cudaError_t cudaMallocHost(void** p, size_t bytes);
cudaError_t cudaFreeHost(void* p);
cudaError_t cudaMemcpy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind);
cudaError_t cudaMemcpyAsync(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s = 0);
cudaError_t cudaMemsetAsync(void* dst, int v, size_t bytes, cudaStream_t s = 0);
cudaError_t cudaStreamSynchronize(cudaStream_t s);
cudaError_t cudaGetLastError(void);
const char* cudaGetErrorString(cudaError_t e);
