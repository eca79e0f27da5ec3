// Matrix-free action of the linear elasticity form
//   a(u, v) = sum_e int_e lambda_e (div u)(div v) + 2 mu_e eps(u):eps(v)
// on a three-component vector H1 space, by the sum factorization of the
// scalar operators (Sec. 4.4) applied to each component, with the components
// coupled only pointwise through the stress (Lines::e3 in k_element.cuh).
#include <type_traits>

#include "fem_internal.h"
#include "k_common.cuh"
#include "k_element.cuh"

namespace {

// Elements per block. Each element holds three slabs (one per component),
// three times the diffusion footprint, and its S3 threads keep the 9 Q
// values of the nine reference-gradient lines in registers; so the block
// keeps at most 256 threads and about 100 KB of shared memory (two blocks
// per SM).
template <typename T, int D1, int Q>
constexpr int ne_elast() {
  constexpr int per = 3 * ElemSmem<T, D1, Q>::SE3 * (int)sizeof(T);
  int ne = 256 / (Q * Q);
  if (ne < 1) ne = 1;
  while (ne > 1 && ne * per > 100 * 1024) --ne;
  return ne;
}

// Resident blocks per SM the kernel is compiled for. The FP32 kernel is
// latency-bound; for p <= 5 it trades registers for up to four resident
// blocks where its shared memory allows (measured at ~4.2e6 vector entries:
// element kernel p = 1 0.590 -> 0.520 ms, p = 2 0.203 -> 0.162, p = 3
// 0.134 -> 0.126, p = 5 0.136 -> 0.097; p = 4 is limited by shared memory,
// and p >= 6 ran 2-4 % slower with the cap, so it keeps the compiler's
// register choice).
template <typename T, int D1, int Q, int NE>
constexpr int elast_min_blocks() {
  if (!std::is_same<T, float>::value || D1 > 6) return 1;
  constexpr int bytes = NE * 3 * ElemSmem<T, D1, Q>::SE3 * (int)sizeof(T);
  constexpr int fit = (227 * 1024) / (bytes + 1024);
  return fit < 4 ? (fit > 0 ? fit : 1) : 4;
}

template <typename T, int D1, int Q, int NE, typename TX>
__global__ void __launch_bounds__(Q * Q * NE, (elast_min_blocks<T, D1, Q, NE>()))
k_elasticity_apply(const int* __restrict__ skip, int ne, int64_t ndof, const int32_t* __restrict__ e2l,
                   const int32_t* __restrict__ pos, const T* __restrict__ Dq, const TX* __restrict__ x,
                   TX* __restrict__ ye) {
  constexpr int NQ = Q * Q * Q, NT = Q * Q * NE;
  if (skip && *skip) return;  // a captured solver iteration after convergence
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x + Q * (threadIdx.y + Q * threadIdx.z);
  const int e0 = blockIdx.x * NE;
  const int nel = min(NE, ne - e0);
  if (tid == 0) l2_prefetch_range(Dq + (size_t)e0 * 12 * NQ, sizeof(T) * (size_t)nel * 12 * NQ);
  elasticity_block<T, D1, Q, NT, TX>(tid, e0, nel, ne, ndof, e2l, Dq, sm, x, ye, pos);
}

template <typename T, int P, int Q, typename TX = T>
fem_status launch(const fem_form* f, const T* D, const TX* x, TX* ye, const int* skip, cudaStream_t s,
                  const int32_t* pos) {
  constexpr int D1 = P + 1, NE = ne_elast<T, D1, Q>();
  const int ne = (int)f->space->ne;
  const size_t bytes = sizeof(T) * (size_t)NE * 3 * ElemSmem<T, D1, Q>::SE3;
  auto kern = k_elasticity_apply<T, D1, Q, NE, TX>;
  if (bytes > 48 * 1024)
    FEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  kern<<<(ne + NE - 1) / NE, dim3(Q, Q, NE), bytes, s>>>(skip, ne, f->space->ndof, f->space->d_e2l, pos, D, x,
                                                         ye);
  FEM_LAUNCHED();
  return FEM_OK;
}

}  // namespace

fem_status fem_elast_tables_init() { return fem_tables_ensure(); }

fem_status fem_launch_apply_elasticity(const fem_form* f, int dtype, const void* x, void* ye, cudaStream_t s,
                                       const int* skip, bool sorted) {
  const int p = f->space->p, q = f->q1d;
  const int32_t* pos = sorted && fem_sorted_evec(f, dtype) ? f->space->d_pos : nullptr;
  if (dtype == FEM_F64) {
#define X(P, Q) \
  if (p == P && q == Q) return launch<double, P, Q>(f, f->d_D, (const double*)x, (double*)ye, skip, s, pos);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else if (dtype == FEM_F32) {
    FEM_TRY(fem_form_ensure_f32(f, s));
#define X(P, Q) \
  if (p == P && q == Q) return launch<float, P, Q>(f, f->d_D32, (const float*)x, (float*)ye, skip, s, pos);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else if (dtype == FEM_DF64) {
    FEM_TRY(fem_form_ensure_df64(f, s));
    const df64* D = reinterpret_cast<const df64*>(f->d_Ddf);
#define X(P, Q) \
  if (p == P && q == Q) return launch<df64, P, Q, double>(f, D, (const double*)x, (double*)ye, skip, s, pos);
    FEM_FOR_EACH_PQ(X)
#undef X
  } else {
    return fem_fail(FEM_EINVAL, "apply: unknown dtype %d", dtype);
  }
  return fem_fail(FEM_EUNSUPPORTED, "apply: (p=%d, q1d=%d) not compiled", p, q);
}
