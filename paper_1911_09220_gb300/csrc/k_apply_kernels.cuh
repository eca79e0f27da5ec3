// Element kernels of the single-problem apply: block shapes, the shared-
// memory plan and the __global__ wrappers around the element operators of
// k_element.cuh. Included by k_apply.cu only.
#pragma once

// Elements per block for a (Q x Q) thread plane: Q^2 * NE fills whole (or
// nearly whole) warps, and the stages with fewer lines pack the lines of all
// NE elements onto full warps. The choice per element type and Q comes from
// measuring both candidates of every order on GB300 (p = 1..8, q = p + 2,
// ~4e6 DOFs, block-packed stages): FP64 takes the larger block except at
// Q = 5, 10; FP32 the smaller one from Q = 5 on (more independent blocks in
// flight on its memory latency); double-float the smaller one at Q = 3, 5, 8.
constexpr int ne_large(int Q) {
  return Q <= 3 ? 32 : Q == 4 ? 16 : Q == 5 ? 5 : Q == 6 ? 8 : Q == 7 ? 5 : Q == 8 ? 4 : 3;
}
constexpr int ne_small(int Q) {
  return Q == 2 ? 16 : Q == 3 ? 14 : Q == 4 ? 8 : Q == 5 ? 10 : Q == 6 ? 4 : Q == 7 ? 2 : Q == 8 ? 2 : Q == 9 ? 1 : 2;
}
// FEM_NE_TABLE (build option): 1 = large for every type, 2 = small for
// every type (the candidate tables of the measurement), else the measured
// choice.
template <typename T>
constexpr int ne_for(int Q) {
#if defined(FEM_NE_TABLE) && FEM_NE_TABLE == 1
  return ne_large(Q);
#elif defined(FEM_NE_TABLE) && FEM_NE_TABLE == 2
  return ne_small(Q);
#endif
  if (std::is_same<T, float>::value) return Q >= 5 ? ne_small(Q) : ne_large(Q);
  if (std::is_same<T, double>::value) return (Q == 5 || Q == 10) ? ne_small(Q) : ne_large(Q);
  return (Q == 3 || Q == 5 || Q == 8) ? ne_small(Q) : ne_large(Q);  // double-float
}

// Shared-memory plan of a block: NE element slabs.
template <typename T, int D1, int Q, int NE>
struct BlockSmem {
  static constexpr size_t bytes = (sizeof(T) * NE * ElemSmem<T, D1, Q>::SE + 15) / 16 * 16;
};

// The block's D range (its elements are consecutive, so the range is one
// contiguous run) is read in stage S3; thread 0 asks the L2 for it at the
// start with one bulk prefetch, so the fetch overlaps the gather and the
// first two contraction stages. (Staging the range into shared memory with a
// bulk copy instead measured slower: the tile lowered the resident blocks
// per SM while the dependent map -> x gather stayed exposed.)
template <typename T, int D1, int Q, int NE, typename TX>
__global__ void __launch_bounds__(Q * Q * NE)
k_diffusion_apply(const int* __restrict__ skip, int ne, const int32_t* __restrict__ e2l, const int32_t* __restrict__ pos,
                  const T* __restrict__ Dq, const TX* __restrict__ x, TX* __restrict__ ye) {
  constexpr int NQ = Q * Q * Q;
  if (skip && *skip) return;  // a captured solver iteration after convergence
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x + Q * (threadIdx.y + Q * threadIdx.z);
  const int e0 = blockIdx.x * NE;
  const int nel = min(NE, ne - e0);
  if (tid == 0) l2_prefetch_range(Dq + (size_t)e0 * 6 * NQ, sizeof(T) * (size_t)nel * 6 * NQ);
  diffusion_block<T, D1, Q, TX>(tid, e0, nel, e2l, Dq, sm, x, ye, pos);
}

template <typename T, int D1, int Q, int NE, typename TX>
__global__ void __launch_bounds__(Q * Q * NE)
k_mass_apply(const int* __restrict__ skip, int ne, const int32_t* __restrict__ e2l, const int32_t* __restrict__ pos,
             const T* __restrict__ Dq, const TX* __restrict__ x, TX* __restrict__ ye) {
  constexpr int NQ = Q * Q * Q;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x + Q * (threadIdx.y + Q * threadIdx.z);
  const int e0 = blockIdx.x * NE;
  const int nel = min(NE, ne - e0);
  if (tid == 0) l2_prefetch_range(Dq + (size_t)e0 * NQ, sizeof(T) * (size_t)nel * NQ);
  mass_block<T, D1, Q, TX>(tid, e0, nel, e2l, Dq, sm, x, ye, pos);
}

template <typename T, int D1, int Q, int NE, typename TX>
__global__ void __launch_bounds__(Q * Q * NE)
k_convection_apply(const int* __restrict__ skip, int ne, const int32_t* __restrict__ e2l, const int32_t* __restrict__ pos,
                   const T* __restrict__ Dq, const TX* __restrict__ x, TX* __restrict__ ye) {
  constexpr int NQ = Q * Q * Q;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x + Q * (threadIdx.y + Q * threadIdx.z);
  const int e0 = blockIdx.x * NE;
  const int nel = min(NE, ne - e0);
  if (tid == 0) l2_prefetch_range(Dq + (size_t)e0 * 3 * NQ, sizeof(T) * (size_t)nel * 3 * NQ);
  convection_block<T, D1, Q, TX>(tid, e0, nel, e2l, Dq, sm, x, ye, pos);
}
