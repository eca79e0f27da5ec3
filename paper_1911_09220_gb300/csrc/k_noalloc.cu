// fem_apply_noalloc: the FP64 operator action y = A x with its E-vector
// scratch in a fixed, library-owned device array instead of memory obtained
// from cudaMalloc.
//
// Who needs this: callers that cannot let the library allocate device memory
// at call time and cannot lend it a scratch buffer either -- for example an
// application whose own memory pool has already reserved (almost) all of the
// GPU's memory, or a latency-critical loop where a cudaMalloc (which may
// synchronise the device and may fail) is not acceptable.
//
// The scratch is a file-scope array of FEM_NOALLOC_MAX_EVEC doubles (32 MiB).
// Every GPU on which this library is loaded holds it until the process exits.
// The kernels are the same element and scatter kernels fem_apply runs; only
// the E-vector pointer differs.
#include <mutex>

#include "fem_internal.h"
#include "k_common.cuh"

#define FEM_NOALLOC_MAX_EVEC (1 << 22)  // E-vector entries: ne * (p+1)^3

namespace {

static __device__ __align__(256) double g_noalloc_evec[FEM_NOALLOC_MAX_EVEC];

// Device address of the array, looked up once per device. In host code the
// symbol name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current.
constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {nullptr};
std::mutex g_addr_mutex;

fem_status noalloc_scratch(double** out) {
  int dev = 0;
  FEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fem_fail(FEM_EUNSUPPORTED, "fem_apply_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_evec);
    if (e != cudaSuccess || !p)
      return fem_fail(FEM_ECUDA, "fem_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = static_cast<double*>(g_addr[dev]);
  return FEM_OK;
}

}  // namespace

extern "C" fem_status fem_apply_noalloc(const fem_form* f, const double* x, double* y, void* stream) {
  if (!f || !x || !y) return fem_fail(FEM_EINVAL, "fem_apply_noalloc: NULL argument");
  if (x == y) return fem_fail(FEM_EINVAL, "fem_apply_noalloc: y must not alias x");
  const int64_t need = f->vdim * f->space->ne * (int64_t)f->space->nd;
  if (need > FEM_NOALLOC_MAX_EVEC)
    return fem_fail(FEM_EINVAL,
                    "fem_apply_noalloc: E-vector of %lld entries (vdim * ne * (p+1)^3) exceeds the fixed scratch of "
                    "%d entries; use fem_apply",
                    (long long)need, FEM_NOALLOC_MAX_EVEC);
  double* ye = nullptr;
  FEM_TRY(noalloc_scratch(&ye));
  cudaStream_t s = (cudaStream_t)stream;
  // The element kernel writes every entry the scatter reads, so the shared
  // array needs no clearing between calls.
  FEM_TRY(fem_launch_apply_element(f, FEM_F64, x, ye, s));
  return fem_launch_scatter(f, FEM_F64, ye, y, nullptr, nullptr, nullptr, 0, s);
}
