// Matrix-free action y = G^T B^T D B G x of the H1 diffusion and mass forms
// (Sec. 4.3, Eq. A = P^T G^T B^T D B G P with P = I) by sum factorization
// (Sec. 4.4: B_ki = B1d_{k1 i1} B1d_{k2 i2} B1d_{k3 i3}, applied one
// direction at a time, O(p^{d+1}) operations per element).
//
// The element operators themselves are in k_element.cuh.
#include <type_traits>

#include "fem_internal.h"
#include "k_common.cuh"
#include "k_element.cuh"
#include "k_apply_kernels.cuh"

namespace {

template <typename K>
fem_status prepare_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) FEM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return FEM_OK;
}

template <typename T, int P, int Q, typename TX = T>
fem_status launch_apply_pq(const fem_form* f, const T* D, const T* B, const T* G, const TX* x, TX* ye,
                           const int* skip, cudaStream_t s, const int32_t* pos) {
  constexpr int D1 = P + 1, NE = ne_for<T>(Q);
  const int ne = (int)f->space->ne;
  const dim3 block(Q, Q, NE);
  const int grid = (ne + NE - 1) / NE;
  (void)B;
  (void)G;
  const size_t bytes = BlockSmem<T, D1, Q, NE>::bytes;
  if (f->kind == FEM_CONVECTION) {
    auto kern = k_convection_apply<T, D1, Q, NE, TX>;
    FEM_TRY(prepare_smem(kern, bytes));
    kern<<<grid, block, bytes, s>>>(skip, ne, f->space->d_e2l, pos, D, x, ye);
  } else if (f->kind == FEM_DIFFUSION) {
    auto kern = k_diffusion_apply<T, D1, Q, NE, TX>;
    FEM_TRY(prepare_smem(kern, bytes));
    kern<<<grid, block, bytes, s>>>(skip, ne, f->space->d_e2l, pos, D, x, ye);
  } else {
    auto kern = k_mass_apply<T, D1, Q, NE, TX>;
    FEM_TRY(prepare_smem(kern, bytes));
    kern<<<grid, block, bytes, s>>>(skip, ne, f->space->d_e2l, pos, D, x, ye);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

// y_i = sum over the inverse map of ye (fixed order: the slots of DOF i in
// increasing (element, local index) order), optional constraint rows
// (y_i = xin_i where mask_i) and per-block partial sums of xin . y. Each
// thread keeps kU DOFs in flight (their off -> idx -> ye load chains are
// independent), the DOFs of one round being kU grid strides apart so that
// every load stays coalesced across the warp. VD = 3: vector entries
// i in [0, 3 ndof), component c = i / ndof of DOF i - c ndof, whose slots
// are read from the E-vector component ye + c * nend.
// sorted: ye is the DOF-sorted E-vector, DOF i's values at ye[off[i] ..
// off[i+1]) (component c's block at ye + c * nend for VD = 3) in the
// inverse map's order: no idx reads, the same sums in the same order.
template <typename T, int VD = 1>
__global__ void k_scatter(const int* __restrict__ skip, int64_t ndof, const int32_t* __restrict__ off,
                          const int32_t* __restrict__ idx, const T* __restrict__ ye, T* __restrict__ y,
                          const uint8_t* __restrict__ mask, const T* __restrict__ xin,
                          double* __restrict__ pdot, int64_t nend = 0, bool sorted = false) {
  constexpr int kU = 4;
  __shared__ double red[32];
  if (skip && *skip) return;
  using A = typename DotAcc<T>::type;
  A acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = VD * ndof;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; base < n; base += stride * kU) {
    int32_t a[kU], b[kU];
    const T* yc[kU];
    int len = 0;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = base + u * stride;
      int64_t li = i;
      yc[u] = ye;
      if (VD > 1) {
        const int c = (i >= ndof) + (i >= 2 * ndof);
        li = i - c * ndof;
        yc[u] = ye + c * nend;
      }
      a[u] = i < n ? __ldg(off + li) : 0;
      b[u] = i < n ? __ldg(off + li + 1) : 0;
      len = max(len, b[u] - a[u]);
    }
    T sum[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) sum[u] = 0;
    if (sorted) {
      for (int j = 0; j < len; ++j) {
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (a[u] + j < b[u]) sum[u] += __ldg(yc[u] + a[u] + j);
      }
    } else {
      for (int j = 0; j < len; ++j) {
        int32_t sl[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) sl[u] = a[u] + j < b[u] ? __ldg(idx + a[u] + j) : -1;
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (sl[u] >= 0) sum[u] += __ldg(yc[u] + sl[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = base + u * stride;
      if (i < n) {
        T v = sum[u];
        if (mask && mask[i]) v = xin[i];
        y[i] = v;
        if (pdot) acc += (A)xin[i] * (A)v;
      }
    }
  }
  if (pdot) {
    const double tot = block_sum((double)acc, red);
    if (threadIdx.x == 0) pdot[blockIdx.x] = tot;
  }
}

template <typename T>
__global__ void k_zero_ess(int64_t ndof, const T* __restrict__ x, const uint8_t* __restrict__ mask,
                           T* __restrict__ xz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof;
       i += (int64_t)gridDim.x * blockDim.x)
    xz[i] = mask[i] ? T(0) : x[i];
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_to_df64(int64_t n, const double* __restrict__ a, df64* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = df64(a[i]);
}

}  // namespace

int fem_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, c = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && c > 0)
      n = c;
    else
      n = 152;
  }
  return n;
}

int fem_kernels_supported(int p, int q1d) {
#define X(P, Q) if (p == P && q1d == Q) return 1;
  FEM_FOR_EACH_PQ(X)
#undef X
  return 0;
}

int fem_scatter_blocks(int64_t ndof) { return grid_for(ndof, 256); }

fem_status fem_apply_tables_init() { return fem_tables_ensure(); }

fem_status fem_form_ensure_f32(const fem_form* fc, cudaStream_t s) {
  fem_form* f = const_cast<fem_form*>(fc);
  if (f->d_D32) return FEM_OK;
  const size_t n = (size_t)f->space->ne * f->ncomp * f->nq;
  FEM_TRY(dev_alloc(&f->d_D32, n + 4));  // 16 bytes of tail padding
  k_to_f32<<<grid_for((int64_t)n, 256), 256, 0, s>>>((int64_t)n, f->d_D, f->d_D32);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_form_ensure_df64(const fem_form* fc, cudaStream_t s) {
  fem_form* f = const_cast<fem_form*>(fc);
  if (f->d_Ddf) return FEM_OK;
  const size_t n = (size_t)f->space->ne * f->ncomp * f->nq;
  FEM_TRY(dev_alloc(&f->d_Ddf, 2 * n + 4));
  k_to_df64<<<grid_for((int64_t)n, 256), 256, 0, s>>>((int64_t)n, f->d_D, reinterpret_cast<df64*>(f->d_Ddf));
  FEM_LAUNCHED();
  return FEM_OK;
}

// The sorted order pays where the E-vector does not stay in L2 between the
// element kernel and the scatter (measured: FP32 diffusion at p = 4 with a
// 131 MB E-vector, scatter 0.110 -> 0.048 ms; FP32 elasticity with 18-25 MB
// E-vectors 3-4 % slower sorted, the pos reads and scattered stores costing
// more than the gathers that hit L2): half the L2 size is the threshold.
bool fem_sorted_evec(const fem_form* f, int dtype) {
  constexpr double kMinBytes = 64.0 * 1024 * 1024;
  const double bytes = (double)f->vdim * f->space->ne * f->space->nd * (dtype == FEM_F32 ? 4 : 8);
  return f->space->mesh->dim == 3 && f->space->d_pos != nullptr && bytes > kMinBytes;
}

fem_status fem_launch_apply_element(const fem_form* f, int dtype, const void* x, void* ye, cudaStream_t s,
                                    const int* skip, bool sorted) {
  if (f->space->mesh->dim == 2) return fem_launch_apply_element_2d(f, dtype, x, ye, s, skip);
  if (f->kind == FEM_ELASTICITY) return fem_launch_apply_elasticity(f, dtype, x, ye, s, skip, sorted);
  const int p = f->space->p, q = f->q1d;
  const int32_t* pos = sorted && fem_sorted_evec(f, dtype) ? f->space->d_pos : nullptr;
  if (dtype == FEM_F64) {
#define X(P, Q)                                                                                            \
  if (p == P && q == Q)                                                                                    \
    return launch_apply_pq<double, P, Q>(f, f->d_D, f->d_B, f->d_G, (const double*)x, (double*)ye, skip, s, pos);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else if (dtype == FEM_F32) {
    FEM_TRY(fem_form_ensure_f32(f, s));
#define X(P, Q)                                                                                            \
  if (p == P && q == Q)                                                                                    \
    return launch_apply_pq<float, P, Q>(f, f->d_D32, f->d_B32, f->d_G32, (const float*)x, (float*)ye, skip, s, pos);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else if (dtype == FEM_DF64) {
    FEM_TRY(fem_form_ensure_df64(f, s));
    const df64* D = reinterpret_cast<const df64*>(f->d_Ddf);
    const df64* B = reinterpret_cast<const df64*>(f->d_Bdf);
    const df64* G = reinterpret_cast<const df64*>(f->d_Gdf);
#define X(P, Q)                                                                                            \
  if (p == P && q == Q)                                                                                    \
    return launch_apply_pq<df64, P, Q, double>(f, D, B, G, (const double*)x, (double*)ye, skip, s, pos);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else {
    return fem_fail(FEM_EINVAL, "apply: unknown dtype %d", dtype);
  }
  return fem_fail(FEM_EUNSUPPORTED, "apply: (p=%d, q1d=%d) not compiled", p, q);
}

fem_status fem_launch_scatter(const fem_form* f, int dtype, const void* ye, void* y, const uint8_t* mask,
                              const void* xin, double* pdot, int nblocks, cudaStream_t s, const int* skip,
                              bool sorted) {
  const fem_space* sp = f->space;
  sorted = sorted && fem_sorted_evec(f, dtype);
  const int grid = nblocks > 0 ? nblocks : fem_scatter_blocks(fem_form_len(f));
  const int64_t nend = sp->ne * (int64_t)sp->nd;
  if (f->vdim == 3) {
    if (dtype == FEM_F64)
      k_scatter<double, 3><<<grid, 256, 0, s>>>(skip, sp->ndof, sp->d_l2e_off, sp->d_l2e_idx, (const double*)ye,
                                                (double*)y, mask, (const double*)xin, pdot, nend, sorted);
    else
      k_scatter<float, 3><<<grid, 256, 0, s>>>(skip, sp->ndof, sp->d_l2e_off, sp->d_l2e_idx, (const float*)ye,
                                               (float*)y, mask, (const float*)xin, pdot, nend, sorted);
  } else if (dtype == FEM_F64) {
    k_scatter<double><<<grid, 256, 0, s>>>(skip, sp->ndof, sp->d_l2e_off, sp->d_l2e_idx, (const double*)ye,
                                           (double*)y, mask, (const double*)xin, pdot, 0, sorted);
  } else {
    k_scatter<float><<<grid, 256, 0, s>>>(skip, sp->ndof, sp->d_l2e_off, sp->d_l2e_idx, (const float*)ye,
                                          (float*)y, mask, (const float*)xin, pdot, 0, sorted);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_zero_ess(const fem_form* f, int dtype, const void* x, void* xz, cudaStream_t s) {
  const int64_t n = fem_form_len(f);
  if (dtype == FEM_F64)
    k_zero_ess<double><<<grid_for(n, 256), 256, 0, s>>>(n, (const double*)x, f->d_ess_mask, (double*)xz);
  else
    k_zero_ess<float><<<grid_for(n, 256), 256, 0, s>>>(n, (const float*)x, f->d_ess_mask, (float*)xz);
  FEM_LAUNCHED();
  return FEM_OK;
}

// ------------------------------------------------------------ public ABI ----
static fem_status ensure_work(fem_form* f, int dtype, size_t n) {
  if (dtype == FEM_F64) {
    if (f->work64_len < n) {
      dev_free(f->d_work64);
      FEM_TRY(dev_alloc(&f->d_work64, n));
      f->work64_len = n;
    }
  } else {
    if (f->work32_len < n) {
      dev_free(f->d_work32);
      FEM_TRY(dev_alloc(&f->d_work32, n));
      f->work32_len = n;
    }
  }
  return FEM_OK;
}

extern "C" fem_status fem_apply_element(const fem_form* f, int dtype, const void* x, void* ye, void* stream) {
  if (!f || !x || !ye) return fem_fail(FEM_EINVAL, "fem_apply_element: NULL argument");
  return fem_launch_apply_element(f, dtype, x, ye, (cudaStream_t)stream);
}

extern "C" fem_status fem_scatter(const fem_form* f, int dtype, const void* ye, void* y, void* stream) {
  if (!f || !ye || !y) return fem_fail(FEM_EINVAL, "fem_scatter: NULL argument");
  if (dtype != FEM_F64 && dtype != FEM_F32 && dtype != FEM_DF64)
    return fem_fail(FEM_EINVAL, "fem_scatter: unknown dtype %d", dtype);
  const int vt = dtype == FEM_F32 ? FEM_F32 : FEM_F64;
  return fem_launch_scatter(f, vt, ye, y, nullptr, nullptr, nullptr, 0, (cudaStream_t)stream);
}

extern "C" fem_status fem_apply(const fem_form* fc, int dtype, const void* x, void* y, int constrained,
                                void* stream) {
  if (!fc || !x || !y) return fem_fail(FEM_EINVAL, "fem_apply: NULL argument");
  if (x == y) return fem_fail(FEM_EINVAL, "fem_apply: y must not alias x");
  if (dtype != FEM_F64 && dtype != FEM_F32 && dtype != FEM_DF64)
    return fem_fail(FEM_EINVAL, "fem_apply: unknown dtype %d", dtype);
  fem_form* f = const_cast<fem_form*>(fc);
  cudaStream_t s = (cudaStream_t)stream;
  const int vt = dtype == FEM_F32 ? FEM_F32 : FEM_F64;  // vector type
  if (constrained && !f->d_ess_mask)
    return fem_fail(FEM_EINVAL, "fem_apply: constrained apply needs fem_form_set_essential");
  void* ye = f->d_ye;  // sized for doubles; float E-vectors use the front half
  if (constrained) {
    FEM_TRY(ensure_work(f, vt, (size_t)fem_form_len(f)));
    void* xz = vt == FEM_F64 ? (void*)f->d_work64 : (void*)f->d_work32;
    FEM_TRY(fem_launch_zero_ess(f, vt, x, xz, s));
    FEM_TRY(fem_launch_apply_element(f, dtype, xz, ye, s, nullptr, true));
    return fem_launch_scatter(f, vt, ye, y, f->d_ess_mask, x, nullptr, 0, s, nullptr, true);
  }
  FEM_TRY(fem_launch_apply_element(f, dtype, x, ye, s, nullptr, true));
  return fem_launch_scatter(f, vt, ye, y, nullptr, nullptr, nullptr, 0, s, nullptr, true);
}
