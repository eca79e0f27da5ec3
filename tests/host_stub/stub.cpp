// Test-only definitions behind tests/host_stub/cuda_runtime.h, and stubs of
// the library's kernel launchers that the host code references but the
// mesh / space tests never reach (they report FEM_EUNSUPPORTED).
#include <cstdlib>
#include <cstring>

#include "fem_internal.h"

cudaError_t cudaMalloc(void** p, size_t bytes) {
  *p = std::malloc(bytes ? bytes : 1);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void* p) {
  std::free(p);
  return cudaSuccess;
}
cudaError_t cudaMallocHost(void** p, size_t bytes) { return cudaMalloc(p, bytes); }
cudaError_t cudaFreeHost(void* p) { return cudaFree(p); }
cudaError_t cudaMemcpy(void* dst, const void* src, size_t bytes, cudaMemcpyKind) {
  std::memmove(dst, src, bytes);
  return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void* dst, const void* src, size_t bytes, cudaMemcpyKind k, cudaStream_t) {
  return cudaMemcpy(dst, src, bytes, k);
}
cudaError_t cudaMemsetAsync(void* dst, int v, size_t bytes, cudaStream_t) {
  std::memset(dst, v, bytes);
  return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
const char* cudaGetErrorString(cudaError_t) { return "host stub"; }

static fem_status no_device() { return fem_fail(FEM_EUNSUPPORTED, "host-only test build: no kernels"); }
fem_status fem_launch_setup(const fem_form*, cudaStream_t) { return no_device(); }
fem_status fem_launch_mark_ess(const fem_form*, cudaStream_t) { return no_device(); }
fem_status fem_launch_dof_coords(const fem_space*, double*, cudaStream_t) { return no_device(); }
fem_status fem_apply_tables_init() { return no_device(); }
fem_status fem_2d_tables_init() { return no_device(); }
fem_status fem_elast_tables_init() { return no_device(); }
int fem_kernels_supported(int, int) { return 0; }

// Test entry to the p-multigrid coarse essential rule (a host function of the
// library without a public ABI): returns the count and, if out is given,
// writes the coarse ids.
extern "C" int64_t test_coarse_essential(const fem_space* sf, const uint8_t* essf, const fem_space* sc,
                                         int32_t* out) {
  const std::vector<int32_t> v = fem_coarse_essential(sf, essf, sc);
  if (out && !v.empty()) std::memcpy(out, v.data(), sizeof(int32_t) * v.size());
  return (int64_t)v.size();
}
