// Matrix-free action y = G^T B^T D B G x of the H1 diffusion and mass forms
// (Sec. 4.3, Eq. A = P^T G^T B^T D B G P with P = I) by sum factorization
// (Sec. 4.4: B_ki = B1d_{k1 i1} B1d_{k2 i2} B1d_{k3 i3}, applied one
// direction at a time, O(p^{d+1}) operations per element).
//
// Element kernel layout: one element per (Q x Q) thread plane, NE elements per
// block. Thread (qx, qy) owns a column of points along z; contractions along x
// and y go through shared memory, contractions along z run in registers.
//   gather   X[z][y][x]          = x_L[e2l[e][z][y][x]]          (G)
//   stage 1  BX, GX  [z][y][qx]  = sum_x B/G[qx][x] X             (B, x)
//   stage 2  bb, gb, bg [z]      = sum_y B/G[qy][y] (BX|GX)       (B, y; registers)
//   stage 3  grad_q              = sum_z B/G[qz][z] (...)         (B, z)
//   point    v_q = D_q grad_q (D symmetric, 6 components)          (D)
//   back z   t0,t1,t2 [dz]      += B/G[qz][dz] v                 (B^T, z)
//   back y   UA, UB [dz][dy][qx] = sum_qy B/G[qy][dy] t           (B^T, y)
//   back x   Y[dz][dy][dx]       = sum_qx G[qx][dx] UA + B[qx][dx] UB (B^T, x)
// Y goes to the E-vector; the scatter kernel sums it into the L-vector
// through the inverse map in a fixed order (atomic-free G^T).
#include "fem_internal.h"
#include "k_common.cuh"

namespace {

// Elements per block for each order: about 128-288 threads per block.
constexpr int ne_per_block(int p) {
  return p == 1 ? 32 : p == 2 ? 16 : p == 3 ? 8 : p == 4 ? 4 : p == 5 ? 4 : 2;
}

template <int D1, int Q>
struct Smem {
  static constexpr int ND = D1 * D1 * D1;
  static constexpr int SA = ND + 2 * D1 * D1 * Q;          // X, BX, GX
  static constexpr int SB = 3 * D1 * Q * Q + 2 * D1 * D1 * Q;  // t0..t2, UA, UB
  static constexpr int SE = SA > SB ? SA : SB;             // per element, in T
};

template <typename T, int D1, int Q, int NE>
__global__ void __launch_bounds__(Q * Q * NE)
k_diffusion_apply(const int* __restrict__ skip, int ne, const int32_t* __restrict__ e2l,
                  const T* __restrict__ Dq, const T* __restrict__ Bg, const T* __restrict__ Gg,
                  const T* __restrict__ x, T* __restrict__ ye) {
  constexpr int ND = D1 * D1 * D1, NQ = Q * Q * Q, SE = Smem<D1, Q>::SE;
  if (skip && *skip) return;  // a captured solver iteration after convergence
  __shared__ T sB[Q * D1], sG[Q * D1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + Q * (ty + Q * tz);
  for (int i = tid; i < Q * D1; i += Q * Q * NE) {
    sB[i] = Bg[i];
    sG[i] = Gg[i];
  }
  const int e = blockIdx.x * NE + tz;
  const bool valid = e < ne;
  T* s = sm + tz * SE;
  T* sX = s;
  T* sBX = s + ND;
  T* sGX = sBX + D1 * D1 * Q;
  if (valid && tx < D1 && ty < D1) {
    const int32_t* map = e2l + (size_t)e * ND;
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      const int k = (z * D1 + ty) * D1 + tx;
      sX[k] = __ldg(x + __ldg(map + k));
    }
  }
  __syncthreads();
  if (ty < D1) {  // stage 1: threads (qx, dy)
    T b[D1], g[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      b[d] = sB[tx * D1 + d];
      g[d] = sG[tx * D1 + d];
    }
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      T u = 0, v = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) {
        const T xv = sX[(z * D1 + ty) * D1 + d];
        u += b[d] * xv;
        v += g[d] * xv;
      }
      sBX[(z * D1 + ty) * Q + tx] = u;
      sGX[(z * D1 + ty) * Q + tx] = v;
    }
  }
  __syncthreads();
  T rbb[D1], rgb[D1], rbg[D1];
  {  // stage 2: threads (qx, qy)
    T b[D1], g[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      b[d] = sB[ty * D1 + d];
      g[d] = sG[ty * D1 + d];
    }
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      T bb = 0, gb = 0, bg = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) {
        const T u = sBX[(z * D1 + d) * Q + tx];
        const T v = sGX[(z * D1 + d) * Q + tx];
        bb += b[d] * u;
        gb += b[d] * v;
        bg += g[d] * u;
      }
      rbb[z] = bb;
      rgb[z] = gb;
      rbg[z] = bg;
    }
  }
  T t0[D1], t1[D1], t2[D1];
#pragma unroll
  for (int d = 0; d < D1; ++d) t0[d] = t1[d] = t2[d] = 0;
  const T* De = Dq + (size_t)(valid ? e : 0) * 6 * NQ + ty * Q + tx;
#pragma unroll 2
  for (int qz = 0; qz < Q; ++qz) {
    T g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      const T bz = sB[qz * D1 + z], gz = sG[qz * D1 + z];
      g0 += bz * rgb[z];
      g1 += bz * rbg[z];
      g2 += gz * rbb[z];
    }
    const int o = qz * Q * Q;
    T d00 = 0, d01 = 0, d02 = 0, d11 = 0, d12 = 0, d22 = 0;
    if (valid) {
      d00 = __ldg(De + 0 * NQ + o);
      d01 = __ldg(De + 1 * NQ + o);
      d02 = __ldg(De + 2 * NQ + o);
      d11 = __ldg(De + 3 * NQ + o);
      d12 = __ldg(De + 4 * NQ + o);
      d22 = __ldg(De + 5 * NQ + o);
    }
    const T v0 = d00 * g0 + d01 * g1 + d02 * g2;
    const T v1 = d01 * g0 + d11 * g1 + d12 * g2;
    const T v2 = d02 * g0 + d12 * g1 + d22 * g2;
#pragma unroll
    for (int d = 0; d < D1; ++d) {
      const T bz = sB[qz * D1 + d], gz = sG[qz * D1 + d];
      t0[d] += bz * v0;
      t1[d] += bz * v1;
      t2[d] += gz * v2;
    }
  }
  __syncthreads();  // phase-A buffers are dead from here on
  T* sT0 = s;
  T* sT1 = sT0 + D1 * Q * Q;
  T* sT2 = sT1 + D1 * Q * Q;
  T* sUA = sT2 + D1 * Q * Q;
  T* sUB = sUA + D1 * D1 * Q;
#pragma unroll
  for (int d = 0; d < D1; ++d) {
    const int k = (d * Q + ty) * Q + tx;
    sT0[k] = t0[d];
    sT1[k] = t1[d];
    sT2[k] = t2[d];
  }
  __syncthreads();
  if (ty < D1) {  // back y: threads (qx, dy)
    T b[Q], g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      b[q] = sB[q * D1 + ty];
      g[q] = sG[q * D1 + ty];
    }
#pragma unroll
    for (int dz = 0; dz < D1; ++dz) {
      T ua = 0, ub = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = (dz * Q + q) * Q + tx;
        ua += b[q] * sT0[k];
        ub += g[q] * sT1[k] + b[q] * sT2[k];
      }
      sUA[(dz * D1 + ty) * Q + tx] = ua;
      sUB[(dz * D1 + ty) * Q + tx] = ub;
    }
  }
  __syncthreads();
  if (valid && tx < D1 && ty < D1) {  // back x: threads (dx, dy)
    T b[Q], g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      b[q] = sB[q * D1 + tx];
      g[q] = sG[q * D1 + tx];
    }
    T* out = ye + (size_t)e * ND;
#pragma unroll
    for (int dz = 0; dz < D1; ++dz) {
      T y = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int k = (dz * D1 + ty) * Q + q;
        y += g[q] * sUA[k] + b[q] * sUB[k];
      }
      out[(dz * D1 + ty) * D1 + tx] = y;
    }
  }
}

// Mass: the same passes with B only and one scalar D per point
// (Sec. 4.4, M_E = B^T D_E B).
template <typename T, int D1, int Q, int NE>
__global__ void __launch_bounds__(Q * Q * NE)
k_mass_apply(const int* __restrict__ skip, int ne, const int32_t* __restrict__ e2l,
             const T* __restrict__ Dq, const T* __restrict__ Bg, const T* __restrict__ x,
             T* __restrict__ ye) {
  constexpr int ND = D1 * D1 * D1, NQ = Q * Q * Q, SE = Smem<D1, Q>::SE;
  if (skip && *skip) return;
  __shared__ T sB[Q * D1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int tid = tx + Q * (ty + Q * tz);
  for (int i = tid; i < Q * D1; i += Q * Q * NE) sB[i] = Bg[i];
  const int e = blockIdx.x * NE + tz;
  const bool valid = e < ne;
  T* s = sm + tz * SE;
  T* sX = s;
  T* sBX = s + ND;
  if (valid && tx < D1 && ty < D1) {
    const int32_t* map = e2l + (size_t)e * ND;
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      const int k = (z * D1 + ty) * D1 + tx;
      sX[k] = __ldg(x + __ldg(map + k));
    }
  }
  __syncthreads();
  if (ty < D1) {
    T b[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) b[d] = sB[tx * D1 + d];
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      T u = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) u += b[d] * sX[(z * D1 + ty) * D1 + d];
      sBX[(z * D1 + ty) * Q + tx] = u;
    }
  }
  __syncthreads();
  T rbb[D1];
  {
    T b[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d) b[d] = sB[ty * D1 + d];
#pragma unroll
    for (int z = 0; z < D1; ++z) {
      T bb = 0;
#pragma unroll
      for (int d = 0; d < D1; ++d) bb += b[d] * sBX[(z * D1 + d) * Q + tx];
      rbb[z] = bb;
    }
  }
  T t0[D1];
#pragma unroll
  for (int d = 0; d < D1; ++d) t0[d] = 0;
  const T* De = Dq + (size_t)(valid ? e : 0) * NQ + ty * Q + tx;
#pragma unroll 2
  for (int qz = 0; qz < Q; ++qz) {
    T u = 0;
#pragma unroll
    for (int z = 0; z < D1; ++z) u += sB[qz * D1 + z] * rbb[z];
    const T v = valid ? __ldg(De + qz * Q * Q) * u : T(0);
#pragma unroll
    for (int d = 0; d < D1; ++d) t0[d] += sB[qz * D1 + d] * v;
  }
  __syncthreads();
  T* sT0 = s;
  T* sUA = sT0 + D1 * Q * Q;
#pragma unroll
  for (int d = 0; d < D1; ++d) sT0[(d * Q + ty) * Q + tx] = t0[d];
  __syncthreads();
  if (ty < D1) {
    T b[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) b[q] = sB[q * D1 + ty];
#pragma unroll
    for (int dz = 0; dz < D1; ++dz) {
      T ua = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) ua += b[q] * sT0[(dz * Q + q) * Q + tx];
      sUA[(dz * D1 + ty) * Q + tx] = ua;
    }
  }
  __syncthreads();
  if (valid && tx < D1 && ty < D1) {
    T b[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) b[q] = sB[q * D1 + tx];
    T* out = ye + (size_t)e * ND;
#pragma unroll
    for (int dz = 0; dz < D1; ++dz) {
      T y = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) y += b[q] * sUA[(dz * D1 + ty) * Q + q];
      out[(dz * D1 + ty) * D1 + tx] = y;
    }
  }
}

template <typename K>
fem_status prepare_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) FEM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return FEM_OK;
}

template <typename T, int P, int Q>
fem_status launch_apply_pq(const fem_form* f, const T* D, const T* B, const T* G, const T* x, T* ye,
                           const int* skip, cudaStream_t s) {
  constexpr int D1 = P + 1, NE = ne_per_block(P);
  const int ne = (int)f->space->ne;
  const dim3 block(Q, Q, NE);
  const int grid = (ne + NE - 1) / NE;
  const size_t bytes = sizeof(T) * NE * Smem<D1, Q>::SE;
  if (f->kind == FEM_DIFFUSION) {
    auto kern = k_diffusion_apply<T, D1, Q, NE>;
    FEM_TRY(prepare_smem(kern, bytes));
    kern<<<grid, block, bytes, s>>>(skip, ne, f->space->d_e2l, D, B, G, x, ye);
  } else {
    auto kern = k_mass_apply<T, D1, Q, NE>;
    FEM_TRY(prepare_smem(kern, bytes));
    kern<<<grid, block, bytes, s>>>(skip, ne, f->space->d_e2l, D, B, x, ye);
  }
  FEM_LAUNCHED();
  return FEM_OK;
}

template <typename T>
__global__ void k_scatter(const int* __restrict__ skip, int64_t ndof, const int32_t* __restrict__ off,
                          const int32_t* __restrict__ idx, const T* __restrict__ ye, T* __restrict__ y,
                          const uint8_t* __restrict__ mask, const T* __restrict__ xin,
                          double* __restrict__ pdot) {
  __shared__ double red[32];
  if (skip && *skip) return;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ndof;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = __ldg(off + i), b = __ldg(off + i + 1);
    T sum = 0;
    for (int32_t k = a; k < b; ++k) sum += __ldg(ye + __ldg(idx + k));
    if (mask && mask[i]) sum = xin[i];
    y[i] = sum;
    if (pdot) acc += (double)xin[i] * (double)sum;
  }
  if (pdot) {
    const double tot = block_sum(acc, red);
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

fem_status fem_form_ensure_f32(const fem_form* fc, cudaStream_t s) {
  fem_form* f = const_cast<fem_form*>(fc);
  if (f->d_D32) return FEM_OK;
  const size_t n = (size_t)f->space->ne * f->ncomp * f->nq;
  FEM_TRY(dev_alloc(&f->d_D32, n));
  k_to_f32<<<grid_for((int64_t)n, 256), 256, 0, s>>>((int64_t)n, f->d_D, f->d_D32);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_apply_element(const fem_form* f, int dtype, const void* x, void* ye, cudaStream_t s,
                                    const int* skip) {
  const int p = f->space->p, q = f->q1d;
  if (dtype == FEM_F64) {
#define X(P, Q)                                                                                            \
  if (p == P && q == Q)                                                                                    \
    return launch_apply_pq<double, P, Q>(f, f->d_D, f->d_B, f->d_G, (const double*)x, (double*)ye, skip, s);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else if (dtype == FEM_F32) {
    FEM_TRY(fem_form_ensure_f32(f, s));
#define X(P, Q)                                                                                            \
  if (p == P && q == Q)                                                                                    \
    return launch_apply_pq<float, P, Q>(f, f->d_D32, f->d_B32, f->d_G32, (const float*)x, (float*)ye, skip, s);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else {
    return fem_fail(FEM_EINVAL, "apply: unknown dtype %d", dtype);
  }
  return fem_fail(FEM_EUNSUPPORTED, "apply: (p=%d, q1d=%d) not compiled", p, q);
}

fem_status fem_launch_scatter(const fem_form* f, int dtype, const void* ye, void* y, const uint8_t* mask,
                              const void* xin, double* pdot, int nblocks, cudaStream_t s, const int* skip) {
  const fem_space* sp = f->space;
  const int grid = nblocks > 0 ? nblocks : fem_scatter_blocks(sp->ndof);
  if (dtype == FEM_F64)
    k_scatter<double><<<grid, 256, 0, s>>>(skip, sp->ndof, sp->d_l2e_off, sp->d_l2e_idx, (const double*)ye,
                                           (double*)y, mask, (const double*)xin, pdot);
  else
    k_scatter<float><<<grid, 256, 0, s>>>(skip, sp->ndof, sp->d_l2e_off, sp->d_l2e_idx, (const float*)ye,
                                          (float*)y, mask, (const float*)xin, pdot);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status fem_launch_zero_ess(const fem_form* f, int dtype, const void* x, void* xz, cudaStream_t s) {
  const int64_t n = f->space->ndof;
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
  if (dtype != FEM_F64 && dtype != FEM_F32) return fem_fail(FEM_EINVAL, "fem_scatter: unknown dtype %d", dtype);
  return fem_launch_scatter(f, dtype, ye, y, nullptr, nullptr, nullptr, 0, (cudaStream_t)stream);
}

extern "C" fem_status fem_apply(const fem_form* fc, int dtype, const void* x, void* y, int constrained,
                                void* stream) {
  if (!fc || !x || !y) return fem_fail(FEM_EINVAL, "fem_apply: NULL argument");
  if (x == y) return fem_fail(FEM_EINVAL, "fem_apply: y must not alias x");
  if (dtype != FEM_F64 && dtype != FEM_F32) return fem_fail(FEM_EINVAL, "fem_apply: unknown dtype %d", dtype);
  fem_form* f = const_cast<fem_form*>(fc);
  cudaStream_t s = (cudaStream_t)stream;
  if (constrained && !f->d_ess_mask)
    return fem_fail(FEM_EINVAL, "fem_apply: constrained apply needs fem_form_set_essential");
  void* ye = f->d_ye;  // sized for doubles; float E-vectors use the front half
  if (constrained) {
    FEM_TRY(ensure_work(f, dtype, (size_t)f->space->ndof));
    void* xz = dtype == FEM_F64 ? (void*)f->d_work64 : (void*)f->d_work32;
    FEM_TRY(fem_launch_zero_ess(f, dtype, x, xz, s));
    FEM_TRY(fem_launch_apply_element(f, dtype, xz, ye, s));
    return fem_launch_scatter(f, dtype, ye, y, f->d_ess_mask, x, nullptr, 0, s);
  }
  FEM_TRY(fem_launch_apply_element(f, dtype, x, ye, s));
  return fem_launch_scatter(f, dtype, ye, y, nullptr, nullptr, nullptr, 0, s);
}
