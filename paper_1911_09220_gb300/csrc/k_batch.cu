// Batched PA operators and Jacobi-PCG over many independent problems (any mix
// of orders, sizes and mass/diffusion forms) with several right-hand sides
// each. The paper has no batched path; this extends its element-parallel
// apply (Sec. 4.3: after G and B the evaluation decouples per element) across
// problems.
//
// Work decomposition: element work items (problem, first element of a tile)
// for the element phase, vector work items (problem, chunk of CH DOFs) for the
// scatter and the CG vector updates. Persistent kernels (grid = SMs x resident
// blocks) stride over the item lists, which are sorted by decreasing cost. An
// element item applies its tile to all nrhs right-hand sides in turn, so each
// D block streams from HBM once and is re-read from L1 / L2 for the other
// right-hand sides. The E-vector is DOF-sorted (each element value at its
// slot's position in the inverse map), so the scatter reads each DOF's
// values contiguously. All launches of an apply (or of `check_every` CG
// iterations) are captured into one CUDA graph and replayed.
//
// System s = (problem i, rhs r) = i * nrhs + r. Batched vectors are
// concatenated problem after problem, problem i's block being [nrhs][ndof_i].
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>
#include <type_traits>

#include "fem_internal.h"
#include "k_common.cuh"
#include "k_element.cuh"
#include "k_element2d.cuh"

namespace {

constexpr int kBT = 256;     // threads of the persistent element / vector blocks
constexpr int kCH = 2048;    // DOFs per vector work item
constexpr int kMaxP = 8;
constexpr int kTiles3 = (kMaxP + 1) * 2;  // tiles[0, kTiles3): hexahedra; then quadrilaterals

struct BProb {
  int p, q, kind, ne, nd, nq, nchunks, sys0;
  int dim;              // 3: hexahedra, 2: quadrilaterals
  int64_t ndof, xoff, yeoff, poff;
  const int32_t* e2l;
  const int32_t* off;
  const int32_t* idx;
  const int32_t* pos;   // DOF-sorted E-vector positions of the slots
  const double* D64;
  const float* D32;
  const double* B64;
  const double* G64;
  const float* B32;
  const float* G32;
  const uint8_t* mask;
  const double* diag64;   // reciprocal Jacobi diagonals (FP64, FP32 copy)
  const float* diag32;
};
struct BItem {
  int prob, e0;
};
struct VItem {
  int prob, chunk;
};

template <typename T>
__device__ __forceinline__ const T* D_of(const BProb& P);
template <>
__device__ __forceinline__ const double* D_of<double>(const BProb& P) { return P.D64; }
template <>
__device__ __forceinline__ const float* D_of<float>(const BProb& P) { return P.D32; }
template <typename T>
__device__ __forceinline__ const T* diag_of(const BProb& P);
template <>
__device__ __forceinline__ const double* diag_of<double>(const BProb& P) { return P.diag64; }
template <>
__device__ __forceinline__ const float* diag_of<float>(const BProb& P) { return P.diag32; }

// Shared-memory slabs a block needs for order p (q = p + 2 or p + 1): one per
// (partial) thread plane of the 256-thread block.
__host__ __device__ constexpr int planes_for(int Q) { return (kBT + Q * Q - 1) / (Q * Q); }
// 2D: one element per row of Q threads.
__host__ __device__ constexpr int rows_for(int Q) { return (kBT + Q - 1) / Q; }

// A 2D tile: rows of Q threads, element el of the tile on row el (tile <=
// floor(256 / Q)), all nrhs right-hand sides in turn; DOF-sorted output.
template <typename T, int D1, int Q>
__device__ __noinline__ void run_tile_2d(const BProb& P, int e0, int tile, int nrhs, const int* __restrict__ done,
                                         const T* __restrict__ X, T* __restrict__ YE, T* sm) {
  constexpr int ND = D1 * D1;
  const int tid = threadIdx.x, el = tid / Q, t = tid % Q;
  const int nel = min(tile, P.ne - e0);
  const T* D = D_of<T>(P);
  for (int r = 0; r < nrhs; ++r) {
    if (done && done[P.sys0 + r]) continue;  // uniform over the block
    const T* x = X + P.xoff + (int64_t)r * P.ndof;
    T* ye = YE + P.yeoff + (int64_t)r * P.ne * ND;
    if (P.kind == FEM_DIFFUSION)
      quad_block<T, D1, Q, T, true>(t, el, e0, nel, P.e2l, D, sm, x, ye, P.pos);
    else
      quad_block<T, D1, Q, T, false>(t, el, e0, nel, P.e2l, D, sm, x, ye, P.pos);
  }
}

template <typename T, int D1, int Q>
__device__ __noinline__ void run_tile(const BProb& P, int e0, int tile, int nrhs, const int* __restrict__ done,
                                      const T* __restrict__ X, T* __restrict__ YE, T* sm) {
  constexpr int ND = D1 * D1 * D1;
  const int tid = threadIdx.x;
  const int nel = min(tile, P.ne - e0);  // tile <= floor(256 / Q^2): whole planes
  const T* D = D_of<T>(P);
  for (int r = 0; r < nrhs; ++r) {
    if (done && done[P.sys0 + r]) continue;  // uniform over the block
    const T* x = X + P.xoff + (int64_t)r * P.ndof;
    T* ye = YE + P.yeoff + (int64_t)r * P.ne * ND;
    if (P.kind == FEM_DIFFUSION)
      diffusion_block<T, D1, Q>(tid, e0, nel, P.e2l, D, sm, x, ye, P.pos);
    else
      mass_block<T, D1, Q>(tid, e0, nel, P.e2l, D, sm, x, ye, P.pos);
  }
}

// Resident blocks per SM the element kernels are compiled for (register
// budget 65536 / (kBT * blocks); the largest variant sets a persistent
// kernel's register count): FP32 4 blocks (64 registers; 16.1 -> 14.6 ms for
// 256 problems x 8 right-hand sides), FP64 2 blocks (128 registers instead
// of 190; 251.2 -> 239.9 ms). Build options FEM_BATCH_MIN_BLOCKS and
// FEM_BATCH_MIN_BLOCKS64.
#ifndef FEM_BATCH_MIN_BLOCKS
#define FEM_BATCH_MIN_BLOCKS 4
#endif
#ifndef FEM_BATCH_MIN_BLOCKS64
#define FEM_BATCH_MIN_BLOCKS64 2
#endif
template <typename T>
constexpr int batch_min_blocks() {
  return std::is_same<T, float>::value ? FEM_BATCH_MIN_BLOCKS : FEM_BATCH_MIN_BLOCKS64;
}

template <typename T>
__global__ void __launch_bounds__(kBT, batch_min_blocks<T>())
k_batch_element(const BProb* __restrict__ probs, const BItem* __restrict__ items, int nitems,
                const int* __restrict__ tiles, int nrhs, const int* __restrict__ done, const T* __restrict__ X,
                T* __restrict__ YE) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem item = items[it];
    const BProb& P = probs[item.prob];
    const int p = P.p, q = P.q;
    __syncthreads();  // the previous item is done with the slabs
    const int tile = tiles[(P.dim == 2 ? kTiles3 : 0) + p * 2 + (q - p - 1)];
    if (P.dim == 2) {
#define CASE(PP, QQ) \
  if (p == PP && q == QQ) run_tile_2d<T, PP + 1, QQ>(P, item.e0, tile, nrhs, done, X, YE, sm);
      FEM_FOR_EACH_PQ_BATCH(CASE)
#undef CASE
    } else {
#define CASE(PP, QQ) \
  if (p == PP && q == QQ) run_tile<T, PP + 1, QQ>(P, item.e0, tile, nrhs, done, X, YE, sm);
      FEM_FOR_EACH_PQ_BATCH(CASE)
#undef CASE
    }
  }
}

// y = G^T ye, optional constraint (y_ess = xin_ess) and partial dot products
// xin . y per (system, chunk). The element kernel writes the E-vector in
// DOF-sorted order (each slot at its position in the inverse map), so DOF
// i's values are ye[off[i] .. off[i+1]) for every right-hand side (ne * nd
// apart); a group of up to kRG right-hand sides shares the offsets. The sums
// run in the inverse map's order.
constexpr int kRG = 8;

template <typename T>
__global__ void __launch_bounds__(kBT)
k_batch_scatter(const BProb* __restrict__ probs, const VItem* __restrict__ items, int nitems, int nrhs,
                const int* __restrict__ done, const T* __restrict__ YE, T* __restrict__ Y, const T* __restrict__ Xin,
                int constrained, double* __restrict__ part) {
  __shared__ double red[32];
  using A = typename DotAcc<T>::type;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const VItem v = items[it];
    const BProb& P = probs[v.prob];
    const int64_t i0 = (int64_t)v.chunk * kCH, i1 = min(i0 + kCH, P.ndof);
    const int64_t es = (int64_t)P.ne * P.nd;  // E-vector stride between right-hand sides
    for (int r0 = 0; r0 < nrhs; r0 += kRG) {
      const int nr = min(kRG, nrhs - r0);
      bool live[kRG];
#pragma unroll
      for (int g = 0; g < kRG; ++g) live[g] = g < nr && !(done && done[P.sys0 + r0 + g]);
      const T* ye = YE + P.yeoff + (int64_t)r0 * es;
      A acc[kRG];
#pragma unroll
      for (int g = 0; g < kRG; ++g) acc[g] = 0;
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int32_t a = P.off[i], b = P.off[i + 1];
        T sum[kRG];
#pragma unroll
        for (int g = 0; g < kRG; ++g) sum[g] = 0;
        for (int32_t k = a; k < b; ++k) {
#pragma unroll
          for (int g = 0; g < kRG; ++g)
            if (live[g]) sum[g] += ye[g * es + k];
        }
        const bool ess = constrained && P.mask && P.mask[i];
#pragma unroll
        for (int g = 0; g < kRG; ++g) {
          if (!live[g]) continue;
          const int64_t xo = P.xoff + (int64_t)(r0 + g) * P.ndof;
          const T sv = ess ? Xin[xo + i] : sum[g];
          Y[xo + i] = sv;
          if (part) acc[g] += (A)Xin[xo + i] * (A)sv;
        }
      }
      if (part) {
        for (int g = 0; g < nr; ++g) {
          if (!live[g]) continue;  // uniform over the block
          const double tot = block_sum((double)acc[g], red);
          if (threadIdx.x == 0) part[P.poff + (int64_t)(r0 + g) * P.nchunks + v.chunk] = tot;
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBT)
k_batch_zero_ess(const BProb* __restrict__ probs, const VItem* __restrict__ items, int nitems, int nrhs,
                 const T* __restrict__ X, T* __restrict__ XZ) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const VItem v = items[it];
    const BProb& P = probs[v.prob];
    const int64_t i0 = (int64_t)v.chunk * kCH, i1 = min(i0 + kCH, P.ndof);
    for (int r = 0; r < nrhs; ++r) {
      const int64_t xo = P.xoff + (int64_t)r * P.ndof;
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
        XZ[xo + i] = (P.mask && P.mask[i]) ? T(0) : X[xo + i];
    }
  }
}

// ------------------------------------------------------------------ CG ----
struct BScal {  // structure of arrays, one entry per system
  double *rz, *alpha, *beta, *rr, *bb, *tol2, *scale;
  int *it, *done, *status, *maxit;
};
enum { ST_RUN = 0, ST_CONV = 1, ST_NOCONV = 2, ST_BREAK = 3 };

__device__ double sys_sum(const double* part, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  return block_sum(v, red);
}

// z = r dinv, p = z; partials r.z, r.r, b.b (b may be null)
template <typename T>
__global__ void __launch_bounds__(kBT)
k_bcg_init(const BProb* __restrict__ probs, const VItem* __restrict__ items, int nitems, int nrhs,
           const int* __restrict__ done, const T* __restrict__ R, T* __restrict__ Z, T* __restrict__ Pv,
           const double* __restrict__ Bv, double* __restrict__ part, int64_t pstride) {
  __shared__ double red[32];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const VItem v = items[it];
    const BProb& P = probs[v.prob];
    const T* dinv = diag_of<T>(P);
    const int64_t i0 = (int64_t)v.chunk * kCH, i1 = min(i0 + kCH, P.ndof);
    for (int r = 0; r < nrhs; ++r) {
      if (done && done[P.sys0 + r]) continue;
      const int64_t xo = P.xoff + (int64_t)r * P.ndof;
      using A = typename DotAcc<T>::type;
      A rz = 0, rr = 0;
      double bb = 0;
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const T ri = R[xo + i];
        const T zi = ri * dinv[i];
        Z[xo + i] = zi;
        Pv[xo + i] = zi;
        rz += (A)ri * (A)zi;
        rr += (A)ri * (A)ri;
        if (Bv) bb += Bv[xo + i] * Bv[xo + i];
      }
      const int64_t slot = P.poff + (int64_t)r * P.nchunks + v.chunk;
      double s = block_sum((double)rz, red);
      if (threadIdx.x == 0) part[slot] = s;
      s = block_sum((double)rr, red);
      if (threadIdx.x == 0) part[pstride + slot] = s;
      s = block_sum(bb, red);
      if (threadIdx.x == 0) part[2 * pstride + slot] = s;
    }
  }
}

// One block per system. bb_given >= 0 replaces b.b (normalised inner solves).
__global__ void k_bcg_init_scalars(const BProb* __restrict__ probs, int nrhs, BScal sc, const double* __restrict__ part,
                                   int64_t pstride, double rtol, double bb_given, int maxit) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  const BProb& P = probs[s / nrhs];
  const int r = s % nrhs;
  if (sc.done[s] == 2) return;  // frozen by the caller (already converged outside)
  const int64_t slot = P.poff + (int64_t)r * P.nchunks;
  const double rz = sys_sum(part + slot, P.nchunks, red);
  const double rr = sys_sum(part + pstride + slot, P.nchunks, red);
  const double bb = sys_sum(part + 2 * pstride + slot, P.nchunks, red);
  if (threadIdx.x == 0) {
    sc.rz[s] = rz;
    sc.rr[s] = rr;
    sc.bb[s] = bb_given >= 0 ? bb_given : bb;
    sc.tol2[s] = rtol * rtol * sc.bb[s];
    sc.it[s] = 0;
    sc.maxit[s] = maxit;
    sc.status[s] = ST_RUN;
    sc.done[s] = 0;
    if (!isfinite(rz) || !isfinite(rr)) {
      sc.done[s] = 1;
      sc.status[s] = ST_BREAK;
    } else if (rr <= sc.tol2[s]) {
      sc.done[s] = 1;
      sc.status[s] = ST_CONV;
    }
  }
}

__global__ void k_bcg_alpha(const BProb* __restrict__ probs, int nrhs, BScal sc, const double* __restrict__ part) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  if (sc.done[s]) return;
  const BProb& P = probs[s / nrhs];
  const int r = s % nrhs;
  const double pq = sys_sum(part + P.poff + (int64_t)r * P.nchunks, P.nchunks, red);
  if (threadIdx.x == 0) {
    if (!(pq > 0.0) || !isfinite(pq)) {
      sc.done[s] = 1;
      sc.status[s] = ST_BREAK;
    } else {
      sc.alpha[s] = sc.rz[s] / pq;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBT)
k_bcg_update(const BProb* __restrict__ probs, const VItem* __restrict__ items, int nitems, int nrhs, BScal sc,
             T* __restrict__ X, T* __restrict__ R, T* __restrict__ Z, const T* __restrict__ Pv,
             const T* __restrict__ Qv, double* __restrict__ part, int64_t pstride) {
  __shared__ double red[32];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const VItem v = items[it];
    const BProb& P = probs[v.prob];
    const T* dinv = diag_of<T>(P);
    const int64_t i0 = (int64_t)v.chunk * kCH, i1 = min(i0 + kCH, P.ndof);
    for (int r = 0; r < nrhs; ++r) {
      const int s = P.sys0 + r;
      if (sc.done[s]) continue;
      const T a = (T)sc.alpha[s];
      const int64_t xo = P.xoff + (int64_t)r * P.ndof;
      using A = typename DotAcc<T>::type;
      A rz = 0, rr = 0;
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        X[xo + i] += a * Pv[xo + i];
        const T ri = R[xo + i] - a * Qv[xo + i];
        R[xo + i] = ri;
        const T zi = ri * dinv[i];
        Z[xo + i] = zi;
        rz += (A)ri * (A)zi;
        rr += (A)ri * (A)ri;
      }
      const int64_t slot = P.poff + (int64_t)r * P.nchunks + v.chunk;
      double t = block_sum((double)rz, red);
      if (threadIdx.x == 0) part[pstride + slot] = t;
      t = block_sum((double)rr, red);
      if (threadIdx.x == 0) part[2 * pstride + slot] = t;
    }
  }
}

__global__ void k_bcg_beta(const BProb* __restrict__ probs, int nrhs, BScal sc, const double* __restrict__ part,
                           int64_t pstride) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  if (sc.done[s]) return;
  const BProb& P = probs[s / nrhs];
  const int r = s % nrhs;
  const int64_t slot = P.poff + (int64_t)r * P.nchunks;
  const double rz = sys_sum(part + pstride + slot, P.nchunks, red);
  const double rr = sys_sum(part + 2 * pstride + slot, P.nchunks, red);
  if (threadIdx.x == 0) {
    sc.it[s] += 1;
    sc.rr[s] = rr;
    if (!isfinite(rz) || !isfinite(rr)) {
      sc.done[s] = 1;
      sc.status[s] = ST_BREAK;
    } else if (rr <= sc.tol2[s]) {
      sc.done[s] = 1;
      sc.status[s] = ST_CONV;
    } else if (sc.it[s] >= sc.maxit[s]) {
      sc.done[s] = 1;
      sc.status[s] = ST_NOCONV;
    } else {
      sc.beta[s] = rz / sc.rz[s];
      sc.rz[s] = rz;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBT)
k_bcg_p(const BProb* __restrict__ probs, const VItem* __restrict__ items, int nitems, int nrhs, BScal sc,
        const T* __restrict__ Z, T* __restrict__ Pv) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const VItem v = items[it];
    const BProb& P = probs[v.prob];
    const int64_t i0 = (int64_t)v.chunk * kCH, i1 = min(i0 + kCH, P.ndof);
    for (int r = 0; r < nrhs; ++r) {
      const int s = P.sys0 + r;
      if (sc.done[s]) continue;
      const T b = (T)sc.beta[s];
      const int64_t xo = P.xoff + (int64_t)r * P.ndof;
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) Pv[xo + i] = Z[xo + i] + b * Pv[xo + i];
    }
  }
}

// r = b - y (FP64), partial r.r per (system, chunk); systems with done == 2
// (frozen) are skipped.
__global__ void __launch_bounds__(kBT)
k_b_residual(const BProb* __restrict__ probs, const VItem* __restrict__ items, int nitems, int nrhs,
             const double* __restrict__ Bv, const double* __restrict__ Yv, double* __restrict__ R,
             double* __restrict__ part) {
  __shared__ double red[32];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const VItem v = items[it];
    const BProb& P = probs[v.prob];
    const int64_t i0 = (int64_t)v.chunk * kCH, i1 = min(i0 + kCH, P.ndof);
    for (int r = 0; r < nrhs; ++r) {
      const int64_t xo = P.xoff + (int64_t)r * P.ndof;
      double rr = 0;
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double ri = Bv[xo + i] - Yv[xo + i];
        R[xo + i] = ri;
        rr += ri * ri;
      }
      const double t = block_sum(rr, red);
      if (threadIdx.x == 0) part[P.poff + (int64_t)r * P.nchunks + v.chunk] = t;
    }
  }
}

// per system: out[s] = sum of its partials
__global__ void k_b_sum(const BProb* __restrict__ probs, int nrhs, const double* __restrict__ part,
                        double* __restrict__ out) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  const BProb& P = probs[s / nrhs];
  const double v = sys_sum(part + P.poff + (int64_t)(s % nrhs) * P.nchunks, P.nchunks, red);
  if (threadIdx.x == 0) out[s] = v;
}

// r32 = r / sqrt(rr_s), x32 = 0 (systems with scale 0 are left at zero)
__global__ void __launch_bounds__(kBT)
k_b_to_f32(const BProb* __restrict__ probs, const VItem* __restrict__ items, int nitems, int nrhs,
           const double* __restrict__ R, const double* __restrict__ rr, float* __restrict__ R32,
           float* __restrict__ X32) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const VItem v = items[it];
    const BProb& P = probs[v.prob];
    const int64_t i0 = (int64_t)v.chunk * kCH, i1 = min(i0 + kCH, P.ndof);
    for (int r = 0; r < nrhs; ++r) {
      const double nr = rr[P.sys0 + r];
      const double inv = nr > 0 ? 1.0 / sqrt(nr) : 0.0;
      const int64_t xo = P.xoff + (int64_t)r * P.ndof;
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        R32[xo + i] = (float)(R[xo + i] * inv);
        X32[xo + i] = 0.0f;
      }
    }
  }
}

__global__ void __launch_bounds__(kBT)
k_b_axpy(const BProb* __restrict__ probs, const VItem* __restrict__ items, int nitems, int nrhs,
         const double* __restrict__ rr, const int* __restrict__ frozen, const float* __restrict__ D32,
         double* __restrict__ X) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const VItem v = items[it];
    const BProb& P = probs[v.prob];
    const int64_t i0 = (int64_t)v.chunk * kCH, i1 = min(i0 + kCH, P.ndof);
    for (int r = 0; r < nrhs; ++r) {
      if (frozen[P.sys0 + r] == 2) continue;
      const double sc = sqrt(rr[P.sys0 + r]);
      const int64_t xo = P.xoff + (int64_t)r * P.ndof;
      for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) X[xo + i] += sc * (double)D32[xo + i];
    }
  }
}

__global__ void k_recip_vec(int64_t n, double* __restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = 1.0 / a[i];
}

__global__ void k_cast_vec(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

template <typename T>
size_t slab_bytes(int p, int q, int dim) {
  if (dim == 2) {
#define X(P, Q) \
  if (p == P && q == Q) return sizeof(T) * (size_t)rows_for(Q) * (size_t)Smem2<P + 1, Q>::SE;
    FEM_FOR_EACH_PQ_BATCH(X)
#undef X
    return 0;
  }
#define X(P, Q) \
  if (p == P && q == Q) return sizeof(T) * (size_t)planes_for(Q) * (size_t)ElemSmem<T, P + 1, Q>::SE;
  FEM_FOR_EACH_PQ_BATCH(X)
#undef X
  return 0;
}

}  // namespace

// ---------------------------------------------------------------- handle ----
struct fem_batch {
  std::vector<const fem_form*> forms;
  int nprob = 0, nrhs = 0;
  std::vector<BProb> hprobs;
  std::vector<int64_t> off;     // prefix sums of ndof
  int64_t len = 0;              // nrhs * sum ndof
  int64_t nsys = 0, pstride = 0;
  int64_t ye_len = 0;
  BProb* d_probs = nullptr;
  BItem* d_items = nullptr;
  int nitems = 0;
  VItem* d_vitems = nullptr;
  int nvitems = 0;
  int* d_tiles = nullptr;       // hexahedra [kMaxP + 1][2], then quadrilaterals: elements per item for (p, q = p+1 / p+2)
  int h_tiles[(kMaxP + 1) * 2];
  int h_tiles2[(kMaxP + 1) * 2];  // quadrilaterals: floor(256 / q) (rows of q threads)
  double* d_ye = nullptr;       // E-vector scratch for all systems (float uses the front half)
  double* d_diag = nullptr;
  float* d_diag32 = nullptr;
  // solver state
  double* d_vec64 = nullptr;    // 7 * len: x, r, z, p, q, t, b-copy
  float* d_vec32 = nullptr;     // 6 * len
  double* d_part = nullptr;     // 3 * pstride
  double* d_sc = nullptr;       // 7 * nsys doubles + 4 * nsys ints
  BScal sc;
  int grid_el64 = 0, grid_el32 = 0, grid_vec = 0;
  size_t smem64 = 0, smem32 = 0;
  // cached apply graph
  cudaGraphExec_t apply_exec = nullptr;
  const void* g_x = nullptr;
  void* g_y = nullptr;
  int g_dtype = -1, g_cons = -1;
};

namespace {

fem_status setup_grids(fem_batch* b) {
  size_t s64 = 0, s32 = 0;
  for (const BProb& P : b->hprobs) {
    s64 = std::max(s64, slab_bytes<double>(P.p, P.q, P.dim));
    s32 = std::max(s32, slab_bytes<float>(P.p, P.q, P.dim));
  }
  b->smem64 = s64;
  b->smem32 = s32;
  FEM_CUDA(cudaFuncSetAttribute(k_batch_element<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64));
  FEM_CUDA(cudaFuncSetAttribute(k_batch_element<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32));
  int n64 = 0, n32 = 0;
  FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n64, k_batch_element<double>, kBT, s64));
  FEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n32, k_batch_element<float>, kBT, s32));
  const int sms = fem_sm_count();
  b->grid_el64 = std::max(1, n64) * sms;
  b->grid_el32 = std::max(1, n32) * sms;
  b->grid_vec = sms * 8;
  return FEM_OK;
}

fem_status build_items(fem_batch* b) {
  // element items, sorted by decreasing cost (element count of the tile x
  // work per element ~ q^4), so the static stride balances
  std::vector<std::pair<double, BItem>> el;
  for (int i = 0; i < b->nprob; ++i) {
    const BProb& P = b->hprobs[i];
    const int tile = (P.dim == 2 ? b->h_tiles2 : b->h_tiles)[P.p * 2 + (P.q - P.p - 1)];
    const double cost = (double)tile * std::pow((double)P.q, P.dim + 1.0) * (P.kind == FEM_DIFFUSION ? 3.0 : 1.0);
    for (int e0 = 0; e0 < P.ne; e0 += tile) el.push_back({cost, BItem{i, e0}});
  }
  std::stable_sort(el.begin(), el.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  std::vector<BItem> items(el.size());
  for (size_t k = 0; k < el.size(); ++k) items[k] = el[k].second;
  dev_free(b->d_items);
  b->nitems = (int)items.size();
  FEM_TRY(dev_alloc(&b->d_items, items.size()));
  FEM_CUDA(cudaMemcpy(b->d_items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice));
  return FEM_OK;
}

fem_status upload_probs(fem_batch* b) {
  FEM_CUDA(cudaMemcpy(b->d_probs, b->hprobs.data(), sizeof(BProb) * b->hprobs.size(), cudaMemcpyHostToDevice));
  FEM_CUDA(cudaMemcpy(b->d_tiles, b->h_tiles, sizeof(b->h_tiles), cudaMemcpyHostToDevice));
  FEM_CUDA(cudaMemcpy(b->d_tiles + kTiles3, b->h_tiles2, sizeof(b->h_tiles2), cudaMemcpyHostToDevice));
  return FEM_OK;
}

template <typename T>
fem_status launch_apply(fem_batch* b, const T* X, T* Y, int constrained, const int* done, double* part, T* xz,
                        cudaStream_t s) {
  const int dt = std::is_same<T, double>::value ? FEM_F64 : FEM_F32;
  const T* xin = X;
  if (constrained) {
    k_batch_zero_ess<T><<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, X, xz);
    xin = xz;
  }
  k_batch_element<T><<<dt == FEM_F64 ? b->grid_el64 : b->grid_el32, kBT, dt == FEM_F64 ? b->smem64 : b->smem32, s>>>(
      b->d_probs, b->d_items, b->nitems, b->d_tiles, b->nrhs, done, xin, (T*)b->d_ye);
  k_batch_scatter<T><<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, done, (T*)b->d_ye,
                                                 Y, X, constrained, part);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status ensure_solver(fem_batch* b, bool mixed, cudaStream_t s) {
  if (!b->d_vec64) FEM_TRY(dev_alloc(&b->d_vec64, (size_t)7 * b->len));
  if (mixed && !b->d_vec32) FEM_TRY(dev_alloc(&b->d_vec32, (size_t)6 * b->len));
  if (!b->d_part) FEM_TRY(dev_alloc(&b->d_part, (size_t)3 * b->pstride));
  if (!b->d_sc) {
    FEM_TRY(dev_alloc(&b->d_sc, (size_t)11 * b->nsys));
    double* d = b->d_sc;
    const int64_t n = b->nsys;
    b->sc.rz = d; b->sc.alpha = d + n; b->sc.beta = d + 2 * n; b->sc.rr = d + 3 * n; b->sc.bb = d + 4 * n;
    b->sc.tol2 = d + 5 * n; b->sc.scale = d + 6 * n;
    int* ip = reinterpret_cast<int*>(d + 7 * n);
    b->sc.it = ip; b->sc.done = ip + n; b->sc.status = ip + 2 * n; b->sc.maxit = ip + 3 * n;
  }
  if (mixed) {
    for (int i = 0; i < b->nprob; ++i) {
      FEM_TRY(fem_form_ensure_f32(b->forms[i], s));
      b->hprobs[i].D32 = b->forms[i]->d_D32;
    }
  }
  return FEM_OK;
}

template <typename T>
fem_status bcg_iteration(fem_batch* b, T* X, T* R, T* Z, T* Pv, T* Qv, T* XZ, cudaStream_t s) {
  FEM_TRY(launch_apply<T>(b, Pv, Qv, 1, b->sc.done, b->d_part, XZ, s));
  k_bcg_alpha<<<(int)b->nsys, 128, 0, s>>>(b->d_probs, b->nrhs, b->sc, b->d_part);
  k_bcg_update<T><<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, b->sc, X, R, Z, Pv, Qv,
                                              b->d_part, b->pstride);
  k_bcg_beta<<<(int)b->nsys, 128, 0, s>>>(b->d_probs, b->nrhs, b->sc, b->d_part, b->pstride);
  k_bcg_p<T><<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, b->sc, Z, Pv);
  FEM_LAUNCHED();
  return FEM_OK;
}

// Iterate until every system is done; graph of `k` iterations replayed.
template <typename T>
fem_status bcg_loop(fem_batch* b, T* X, T* R, T* Z, T* Pv, T* Qv, T* XZ, const fem_solve_opts& o, int maxit,
                    cudaStream_t s) {
  const int k = o.check_every > 0 ? o.check_every : 16;
  cudaGraphExec_t exec = nullptr;
  if (o.use_graph) {
    cudaStream_t cs;
    FEM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    fem_status st = FEM_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = fem_fail(FEM_ECUDA, "batch solve: capture failed to begin");
    } else {
      for (int i = 0; i < k && st == FEM_OK; ++i) st = bcg_iteration<T>(b, X, R, Z, Pv, Qv, XZ, cs);
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (st == FEM_OK && e != cudaSuccess) st = fem_fail(FEM_ECUDA, "batch solve: end capture: %s", cudaGetErrorString(e));
    }
    if (st == FEM_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "batch solve: graph instantiation failed");
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != FEM_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      return st;
    }
  }
  std::vector<int> hdone(b->nsys);
  fem_status st = FEM_OK;
  const int rounds = maxit / k + 2;
  for (int round = 0; round < rounds; ++round) {
    if (exec) {
      if (cudaGraphLaunch(exec, s) != cudaSuccess) {
        st = fem_fail(FEM_ECUDA, "batch solve: graph launch failed");
        break;
      }
    } else {
      for (int i = 0; i < k && st == FEM_OK; ++i) st = bcg_iteration<T>(b, X, R, Z, Pv, Qv, XZ, s);
      if (st != FEM_OK) break;
    }
    if (cudaMemcpyAsync(hdone.data(), b->sc.done, sizeof(int) * b->nsys, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = fem_fail(FEM_ECUDA, "batch solve: status read failed");
      break;
    }
    bool all = true;
    for (int v : hdone) all = all && (v != 0);
    if (all) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  return st;
}

}  // namespace

fem_status fem_batch_tables_init() { return fem_tables_ensure(); }

extern "C" fem_status fem_batch_create(const fem_form* const* forms, int nprob, int nrhs, void* stream,
                                       fem_batch** out) {
  if (!out || !forms || nprob <= 0 || nrhs <= 0) return fem_fail(FEM_EINVAL, "fem_batch_create: bad arguments");
  *out = nullptr;
  FEM_TRY(fem_batch_tables_init());
  fem_batch* b = new fem_batch();
  b->nprob = nprob;
  b->nrhs = nrhs;
  b->forms.assign(forms, forms + nprob);
  for (int p = 0; p <= kMaxP; ++p)
    for (int j = 0; j < 2; ++j) {
      const int q = p + 1 + j;
      b->h_tiles[p * 2 + j] = std::max(1, kBT / std::max(1, q * q));
      b->h_tiles2[p * 2 + j] = std::max(1, kBT / std::max(1, q));
    }
  int64_t ndof_sum = 0, ye_sum = 0, chunk_sum = 0;
  std::vector<VItem> vitems;
  b->off.push_back(0);
  for (int i = 0; i < nprob; ++i) {
    const fem_form* f = forms[i];
    if (!f) {
      delete b;
      return fem_fail(FEM_EINVAL, "fem_batch_create: form %d is NULL", i);
    }
    const fem_space* sp = f->space;
    if (f->kind == FEM_CONVECTION) {
      delete b;
      return fem_fail(FEM_EUNSUPPORTED, "fem_batch_create: form %d is a convection form", i);
    }
    if (f->kind == FEM_ELASTICITY) {
      delete b;
      return fem_fail(FEM_EINVAL, "fem_batch_create: form %d is an elasticity form", i);
    }

    if (sp->p > 6) {
      delete b;
      return fem_fail(FEM_EUNSUPPORTED, "fem_batch_create: form %d has p = %d; batches hold p <= 6", i, sp->p);
    }
    BProb P{};
    P.p = sp->p; P.q = f->q1d; P.kind = f->kind; P.ne = (int)sp->ne; P.nd = sp->nd; P.nq = f->nq;
    P.dim = sp->mesh->dim;
    P.ndof = sp->ndof;
    P.nchunks = (int)((sp->ndof + kCH - 1) / kCH);
    P.sys0 = i * nrhs;
    P.xoff = (int64_t)nrhs * ndof_sum;
    P.yeoff = (int64_t)nrhs * ye_sum;
    P.poff = (int64_t)nrhs * chunk_sum;
    P.e2l = sp->d_e2l; P.off = sp->d_l2e_off; P.idx = sp->d_l2e_idx; P.pos = sp->d_pos;
    P.D64 = f->d_D; P.D32 = f->d_D32;
    P.B64 = f->d_B; P.G64 = f->d_G; P.B32 = f->d_B32; P.G32 = f->d_G32;
    P.mask = f->d_ess_mask;
    for (int c = 0; c < P.nchunks; ++c) vitems.push_back(VItem{i, c});
    ndof_sum += sp->ndof;
    ye_sum += sp->ne * (int64_t)sp->nd;
    chunk_sum += P.nchunks;
    b->off.push_back(ndof_sum);
    b->hprobs.push_back(P);
  }
  b->len = (int64_t)nrhs * ndof_sum;
  b->nsys = (int64_t)nrhs * nprob;
  b->pstride = (int64_t)nrhs * chunk_sum;
  b->ye_len = (int64_t)nrhs * ye_sum;
  fem_status st = dev_alloc(&b->d_probs, (size_t)nprob);
  if (st == FEM_OK) st = dev_alloc(&b->d_tiles, (size_t)2 * kTiles3);
  if (st == FEM_OK) st = dev_alloc(&b->d_ye, (size_t)b->ye_len);
  if (st == FEM_OK) st = dev_alloc(&b->d_vitems, vitems.size());
  if (st == FEM_OK) {
    b->nvitems = (int)vitems.size();
    if (cudaMemcpy(b->d_vitems, vitems.data(), sizeof(VItem) * vitems.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "fem_batch_create: upload failed");
  }
  if (st == FEM_OK) st = upload_probs(b);
  if (st == FEM_OK) st = build_items(b);
  if (st == FEM_OK) st = setup_grids(b);
  if (st != FEM_OK) {
    fem_batch_destroy(b);
    return st;
  }
  (void)stream;
  *out = b;
  return FEM_OK;
}

extern "C" void fem_batch_destroy(fem_batch* b) {
  if (!b) return;
  if (b->apply_exec) cudaGraphExecDestroy(b->apply_exec);
  dev_free(b->d_probs);
  dev_free(b->d_items);
  dev_free(b->d_vitems);
  dev_free(b->d_tiles);
  dev_free(b->d_ye);
  dev_free(b->d_diag);
  dev_free(b->d_diag32);
  dev_free(b->d_vec64);
  dev_free(b->d_vec32);
  dev_free(b->d_part);
  dev_free(b->d_sc);
  delete b;
}

extern "C" fem_status fem_batch_info(const fem_batch* b, int64_t* total_len, int64_t* off_host) {
  if (!b) return fem_fail(FEM_EINVAL, "fem_batch_info: NULL batch");
  if (total_len) *total_len = b->len;
  if (off_host) std::memcpy(off_host, b->off.data(), sizeof(int64_t) * b->off.size());
  return FEM_OK;
}

extern "C" fem_status fem_batch_apply(fem_batch* b, int dtype, const void* X, void* Y, int constrained,
                                      void* stream) {
  if (!b || !X || !Y) return fem_fail(FEM_EINVAL, "fem_batch_apply: NULL argument");
  if (X == Y) return fem_fail(FEM_EINVAL, "fem_batch_apply: Y must not alias X");
  if (dtype != FEM_F64 && dtype != FEM_F32) return fem_fail(FEM_EINVAL, "fem_batch_apply: unknown dtype");
  cudaStream_t s = (cudaStream_t)stream;
  if (constrained) {
    for (int i = 0; i < b->nprob; ++i) {
      if (!b->forms[i]->d_ess_mask)
        return fem_fail(FEM_EINVAL, "fem_batch_apply: constrained apply needs essential DOFs on every form");
      if (b->hprobs[i].mask != b->forms[i]->d_ess_mask) {
        b->hprobs[i].mask = b->forms[i]->d_ess_mask;
        FEM_TRY(upload_probs(b));
      }
    }
  }
  if (dtype == FEM_F32) {
    bool changed = false;
    for (int i = 0; i < b->nprob; ++i) {
      FEM_TRY(fem_form_ensure_f32(b->forms[i], s));
      if (b->hprobs[i].D32 != b->forms[i]->d_D32) {
        b->hprobs[i].D32 = b->forms[i]->d_D32;
        changed = true;
      }
    }
    if (changed) FEM_TRY(upload_probs(b));
  }
  // constrained applies need a zeroed copy of X: use the front of the solver
  // vectors (allocated on first use)
  void* xz = nullptr;
  if (constrained) {
    if (dtype == FEM_F64) {
      if (!b->d_vec64) FEM_TRY(dev_alloc(&b->d_vec64, (size_t)7 * b->len));
      xz = b->d_vec64 + 5 * b->len;
    } else {
      if (!b->d_vec32) FEM_TRY(dev_alloc(&b->d_vec32, (size_t)6 * b->len));
      xz = b->d_vec32 + 5 * b->len;
    }
  }
  // one CUDA graph per (X, Y, dtype, constrained), re-captured when they change
  if (!b->apply_exec || b->g_x != X || b->g_y != Y || b->g_dtype != dtype || b->g_cons != constrained) {
    if (b->apply_exec) cudaGraphExecDestroy(b->apply_exec);
    b->apply_exec = nullptr;
    cudaStream_t cs;
    FEM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    fem_status st = FEM_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = fem_fail(FEM_ECUDA, "fem_batch_apply: capture failed to begin");
    } else {
      if (dtype == FEM_F64)
        st = launch_apply<double>(b, (const double*)X, (double*)Y, constrained, nullptr, nullptr, (double*)xz, cs);
      else
        st = launch_apply<float>(b, (const float*)X, (float*)Y, constrained, nullptr, nullptr, (float*)xz, cs);
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (st == FEM_OK && e != cudaSuccess) st = fem_fail(FEM_ECUDA, "fem_batch_apply: end capture failed");
    }
    if (st == FEM_OK && cudaGraphInstantiate(&b->apply_exec, g, 0) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "fem_batch_apply: graph instantiation failed");
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != FEM_OK) return st;
    b->g_x = X;
    b->g_y = Y;
    b->g_dtype = dtype;
    b->g_cons = constrained;
  }
  FEM_CUDA(cudaGraphLaunch(b->apply_exec, s));
  return FEM_OK;
}

extern "C" fem_status fem_batch_solve(fem_batch* b, const double* Bv, double* Xv, const fem_solve_opts* opts,
                                      int* iters_host, double* relres_host, void* stream) {
  if (!b || !Bv || !Xv) return fem_fail(FEM_EINVAL, "fem_batch_solve: NULL argument");
  fem_solve_opts o;
  fem_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0) || o.maxit <= 0) return fem_fail(FEM_EINVAL, "fem_batch_solve: rtol > 0 and maxit > 0 required");
  if (o.precond != FEM_PC_JACOBI) return fem_fail(FEM_EUNSUPPORTED, "fem_batch_solve: Jacobi preconditioner only");
  o.inner_rtol = fem_inner_rtol(o, 2);
  const bool mixed = o.precision == FEM_SOLVE_MIXED;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < b->nprob; ++i)
    if (!b->forms[i]->d_ess_mask)
      return fem_fail(FEM_EINVAL, "fem_batch_solve: set essential DOFs (possibly none) on every form first");
  FEM_TRY(ensure_solver(b, mixed, s));
  // constrained diagonals, per problem (shared by its right-hand sides)
  if (!b->d_diag) FEM_TRY(dev_alloc(&b->d_diag, (size_t)b->off.back()));
  if (mixed && !b->d_diag32) FEM_TRY(dev_alloc(&b->d_diag32, (size_t)b->off.back()));
  for (int i = 0; i < b->nprob; ++i) {
    FEM_TRY(fem_assemble_diagonal(b->forms[i], b->d_diag + b->off[i], 1, s));
    b->hprobs[i].diag64 = b->d_diag + b->off[i];
    b->hprobs[i].diag32 = mixed ? b->d_diag32 + b->off[i] : nullptr;
    b->hprobs[i].mask = b->forms[i]->d_ess_mask;
  }
  // the reciprocal diagonals (every iteration multiplies; FP64 divisions per
  // entry bound the FP64 vector updates on GB300's FP64 pipe)
  k_recip_vec<<<grid_for(b->off.back(), 256), 256, 0, s>>>(b->off.back(), b->d_diag);
  FEM_LAUNCHED();
  if (mixed) {
    k_cast_vec<<<grid_for(b->off.back(), 256), 256, 0, s>>>(b->off.back(), b->d_diag, b->d_diag32);
    FEM_LAUNCHED();
  }
  FEM_TRY(upload_probs(b));
  if (b->apply_exec) {  // the problem table changed under the cached graph's kernels: re-capture next time
    cudaGraphExecDestroy(b->apply_exec);
    b->apply_exec = nullptr;
  }
  const int64_t L = b->len, ns = b->nsys;
  double* x = b->d_vec64;
  double* r = x + L;
  double* z = x + 2 * L;
  double* pv = x + 3 * L;
  double* qv = x + 4 * L;
  double* xz = x + 5 * L;
  double* bb = x + 6 * L;
  FEM_CUDA(cudaMemcpyAsync(x, Xv, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
  FEM_CUDA(cudaMemcpyAsync(bb, Bv, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
  // ||b||^2 per system
  std::vector<double> hbb(ns), hrr(ns);
  std::vector<int> hit(ns, 0), hdone(ns, 0), hst(ns, 0), frozen(ns, 0);
  k_bcg_init<double><<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, nullptr, bb, z, pv, bb,
                                                 b->d_part, b->pstride);
  k_b_sum<<<(int)ns, 128, 0, s>>>(b->d_probs, b->nrhs, b->d_part + 2 * b->pstride, b->sc.bb);
  FEM_LAUNCHED();
  FEM_CUDA(cudaMemcpyAsync(hbb.data(), b->sc.bb, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  std::vector<int> total_it(ns, 0);
  int outer = 0;
  fem_status result = FEM_OK;
  for (;;) {
    // true residual r = b - A_c x in FP64 for every system
    FEM_TRY(launch_apply<double>(b, x, qv, 1, nullptr, nullptr, xz, s));
    k_b_residual<<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, bb, qv, r, b->d_part);
    k_b_sum<<<(int)ns, 128, 0, s>>>(b->d_probs, b->nrhs, b->d_part, b->sc.scale);
    FEM_LAUNCHED();
    FEM_CUDA(cudaMemcpyAsync(hrr.data(), b->sc.scale, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    bool all = true, any_bad = false;
    for (int64_t k = 0; k < ns; ++k) {
      const double tol2 = o.rtol * o.rtol * hbb[k];
      frozen[k] = (hrr[k] <= tol2 || !(hbb[k] > 0)) ? 2 : 0;
      if (!std::isfinite(hrr[k])) any_bad = true;
      if (frozen[k] != 2) all = false;
    }
    if (all || any_bad) {
      if (any_bad) result = fem_fail(FEM_EBREAKDOWN, "fem_batch_solve: non-finite residual");
      break;
    }
    int maxtot = 0;
    for (int64_t k = 0; k < ns; ++k) maxtot = std::max(maxtot, total_it[k]);
    if (maxtot >= o.maxit || outer >= o.max_outer) {
      result = fem_fail(FEM_ENOCONV, "fem_batch_solve: not every system converged (%d iterations)", maxtot);
      break;
    }
    FEM_CUDA(cudaMemcpyAsync(b->sc.done, frozen.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    const int maxit_in = o.maxit - maxtot;
    if (!mixed) {
      k_bcg_init<double><<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, b->sc.done, r, z,
                                                     pv, nullptr, b->d_part, b->pstride);
      k_bcg_init_scalars<<<(int)ns, 128, 0, s>>>(b->d_probs, b->nrhs, b->sc, b->d_part, b->pstride, o.rtol, -1.0,
                                                 maxit_in);
      FEM_LAUNCHED();
      // tol relative to ||b||: bb holds r.r of the restart; set it to ||b||^2
      FEM_CUDA(cudaMemcpyAsync(b->sc.bb, hbb.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
      std::vector<double> tol2(ns);
      for (int64_t k = 0; k < ns; ++k) tol2[k] = o.rtol * o.rtol * hbb[k];
      FEM_CUDA(cudaMemcpyAsync(b->sc.tol2, tol2.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
      FEM_TRY(bcg_loop<double>(b, x, r, z, pv, qv, xz, o, maxit_in, s));
    } else {
      float* x32 = b->d_vec32;
      float* r32 = x32 + L;
      float* z32 = x32 + 2 * L;
      float* p32 = x32 + 3 * L;
      float* q32 = x32 + 4 * L;
      float* xz32 = x32 + 5 * L;
      k_b_to_f32<<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, r, b->sc.scale, r32, x32);
      k_bcg_init<float><<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, b->sc.done, r32, z32,
                                                    p32, nullptr, b->d_part, b->pstride);
      k_bcg_init_scalars<<<(int)ns, 128, 0, s>>>(b->d_probs, b->nrhs, b->sc, b->d_part, b->pstride, o.inner_rtol, 1.0,
                                                 maxit_in);
      FEM_LAUNCHED();
      // a system whose pass needs less than inner_rtol to reach the tolerance
      // stops at half of it (tolerances of the normalised inner systems)
      std::vector<double> tol2(ns);
      for (int64_t k = 0; k < ns; ++k) {
        const double need = hrr[k] > 0 ? 0.25 * o.rtol * o.rtol * hbb[k] / hrr[k] : 0.0;
        tol2[k] = std::max(o.inner_rtol * o.inner_rtol, need);
      }
      FEM_CUDA(cudaMemcpyAsync(b->sc.tol2, tol2.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
      FEM_TRY(bcg_loop<float>(b, x32, r32, z32, p32, q32, xz32, o, maxit_in, s));
      FEM_CUDA(cudaMemcpyAsync(b->sc.done, frozen.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
      k_b_axpy<<<b->grid_vec, kBT, 0, s>>>(b->d_probs, b->d_vitems, b->nvitems, b->nrhs, b->sc.scale, b->sc.done, x32,
                                           x);
      FEM_LAUNCHED();
    }
    FEM_CUDA(cudaMemcpyAsync(hit.data(), b->sc.it, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaMemcpyAsync(hst.data(), b->sc.status, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    for (int64_t k = 0; k < ns; ++k)
      if (frozen[k] != 2) total_it[k] += hit[k];
    bool brk = false;
    for (int64_t k = 0; k < ns; ++k) brk = brk || (frozen[k] != 2 && hst[k] == ST_BREAK);
    if (brk) {
      result = fem_fail(FEM_EBREAKDOWN, "fem_batch_solve: CG breakdown in a system");
      break;
    }
    ++outer;
  }
  FEM_CUDA(cudaMemcpyAsync(Xv, x, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  if (iters_host) std::memcpy(iters_host, total_it.data(), sizeof(int) * ns);
  if (relres_host)
    for (int64_t k = 0; k < ns; ++k) relres_host[k] = hbb[k] > 0 ? std::sqrt(hrr[k] / hbb[k]) : 0.0;
  return result;
}

// ---------------------------------------------------------------- tuner ----
// Autotuner: for every (p, q) in the batch, time the batched apply with
// candidate element tiles (elements per work item: the block's maximum
// floor(256 / q^2) and smaller values) by coordinate descent, keep the
// fastest, and cache the result per device name and dtype in a small JSON
// file of lines `{"key": "<device>|<dtype>|p<p>q<q>", "tile": n}`.
extern "C" fem_status fem_batch_tune(fem_batch* b, int dtype, const char* cache_path, void* stream) {
  if (!b) return fem_fail(FEM_EINVAL, "fem_batch_tune: NULL batch");
  if (dtype != FEM_F64 && dtype != FEM_F32) return fem_fail(FEM_EINVAL, "fem_batch_tune: unknown dtype");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaDeviceProp prop;
  FEM_CUDA(cudaGetDevice(&dev));
  FEM_CUDA(cudaGetDeviceProperties(&prop, dev));
  std::string devname = prop.name;
  for (char& c : devname)
    if (c == '"' || c == '|') c = '_';
  const char* dts = dtype == FEM_F64 ? "f64" : "f32";
  std::map<std::string, int> cache;
  if (cache_path) {
    if (FILE* fp = std::fopen(cache_path, "r")) {
      char line[512];
      while (std::fgets(line, sizeof line, fp)) {
        char key[400];
        int tile = 0;
        if (std::sscanf(line, " {\"key\": \"%399[^\"]\", \"tile\": %d}", key, &tile) == 2 && tile > 0) cache[key] = tile;
      }
      std::fclose(fp);
    }
  }
  std::vector<std::pair<int, int>> pqs;
  for (const BProb& P : b->hprobs)  // hexahedral problems (quadrilaterals keep floor(256 / q))
    if (P.dim == 3 && std::find(pqs.begin(), pqs.end(), std::make_pair(P.p, P.q)) == pqs.end())
      pqs.push_back({P.p, P.q});
  auto keyof = [&](int p, int q) { return devname + "|" + dts + "|p" + std::to_string(p) + "q" + std::to_string(q); };
  bool all_cached = true;
  for (auto& pq : pqs) {
    auto it = cache.find(keyof(pq.first, pq.second));
    // a cached tile is clamped to the block's whole planes: every element of
    // a tile needs its plane of q^2 threads among the block's 256
    if (it != cache.end())
      b->h_tiles[pq.first * 2 + (pq.second - pq.first - 1)] =
          std::min(it->second, std::max(1, kBT / (pq.second * pq.second)));
    else
      all_cached = false;
  }
  if (!all_cached) {
    // scratch vectors for timing
    const size_t es = dtype == FEM_F64 ? sizeof(double) : sizeof(float);
    void* X = nullptr;
    void* Y = nullptr;
    FEM_CUDA(cudaMalloc(&X, es * b->len));
    FEM_CUDA(cudaMalloc(&Y, es * b->len));
    FEM_CUDA(cudaMemsetAsync(X, 0, es * b->len, s));
    if (dtype == FEM_F32)
      for (int i = 0; i < b->nprob; ++i) {
        FEM_TRY(fem_form_ensure_f32(b->forms[i], s));
        b->hprobs[i].D32 = b->forms[i]->d_D32;
      }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_apply = [&](float* ms) -> fem_status {
      FEM_TRY(upload_probs(b));
      FEM_TRY(build_items(b));
      for (int w = 0; w < 2; ++w) {
        if (dtype == FEM_F64) FEM_TRY(launch_apply<double>(b, (double*)X, (double*)Y, 0, nullptr, nullptr, nullptr, s));
        else FEM_TRY(launch_apply<float>(b, (float*)X, (float*)Y, 0, nullptr, nullptr, nullptr, s));
      }
      cudaEventRecord(e0, s);
      for (int w = 0; w < 3; ++w) {
        if (dtype == FEM_F64) FEM_TRY(launch_apply<double>(b, (double*)X, (double*)Y, 0, nullptr, nullptr, nullptr, s));
        else FEM_TRY(launch_apply<float>(b, (float*)X, (float*)Y, 0, nullptr, nullptr, nullptr, s));
      }
      cudaEventRecord(e1, s);
      FEM_CUDA(cudaEventSynchronize(e1));
      cudaEventElapsedTime(ms, e0, e1);
      return FEM_OK;
    };
    float best = 0;
    FEM_TRY(time_apply(&best));
    for (auto& pq : pqs) {
      const int slot = pq.first * 2 + (pq.second - pq.first - 1);
      if (cache.count(keyof(pq.first, pq.second))) continue;
      const int tmax = std::max(1, kBT / (pq.second * pq.second));
      int best_tile = b->h_tiles[slot];
      for (int cand = tmax; cand >= std::max(1, tmax / 2); --cand) {
        if (cand == best_tile) continue;
        b->h_tiles[slot] = cand;
        float ms = 0;
        FEM_TRY(time_apply(&ms));
        if (ms < best) {
          best = ms;
          best_tile = cand;
        }
      }
      b->h_tiles[slot] = best_tile;
      cache[keyof(pq.first, pq.second)] = best_tile;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(X);
    cudaFree(Y);
    if (cache_path) {
      if (FILE* fp = std::fopen(cache_path, "w")) {
        for (auto& kv : cache) std::fprintf(fp, "{\"key\": \"%s\", \"tile\": %d}\n", kv.first.c_str(), kv.second);
        std::fclose(fp);
      }
    }
  }
  FEM_TRY(upload_probs(b));
  FEM_TRY(build_items(b));
  if (b->apply_exec) {
    cudaGraphExecDestroy(b->apply_exec);
    b->apply_exec = nullptr;
  }
  return FEM_OK;
}

extern "C" fem_status fem_batch_tiles(const fem_batch* b, int* tiles_host) {
  if (!b || !tiles_host) return fem_fail(FEM_EINVAL, "fem_batch_tiles: NULL argument");
  std::memcpy(tiles_host, b->h_tiles, sizeof(b->h_tiles));
  return FEM_OK;
}
