// Jacobi-preconditioned conjugate gradients on the partially assembled
// operator (Sec. 5.2: CGSolver with a relative tolerance and an iteration cap;
// Sec. 4.4: with PA there are no matrix entries, so the preconditioner is the
// assembled diagonal), FP64 or FP32-inner / FP64-outer iterative refinement.
//
// One iteration is four launches on the solver stream:
//   element kernel (p -> E-vector), scatter (q = A_c p, partials of p.q),
//   update (every block sums the p.q partials to alpha; x += a p, r -= a q,
//   z = r dinv, partials of r.z and r.r), direction (every block sums the
//   r.z and r.r partials: convergence test, beta; p = z + beta p).
// The scalar steps run redundantly in every block from the same partials in
// the same order, so every block takes the same decision and no single-block
// kernel sits between the vector kernels; block 0 alone writes the solver
// state, into fields no other block of that launch reads (r.z alternates
// between two slots by iteration parity). Scalars live in device memory;
// every kernel returns at once when the device `done` word is set, so a CUDA
// graph of `check_every` iterations can be replayed and the host only polls
// between replays. Reductions are block partials summed in a fixed order:
// results are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "fem_internal.h"
#include "k_common.cuh"

namespace {

struct CgScalars {
  double rzb[2];    // r.z of the current residual in slot it & 1
  double beta, rr, bb, tol2;
  double upd2;      // reliable updates: stop for an FP64 update once r.r <= upd2
  double rz_new;    // r.z of the iteration that stopped for an update
  int it, done, status, maxit;  // read by the host as four ints
  int it1;          // it + 1, written by the update kernel for its last block
  int ru;           // 1: reliable-update mode
  unsigned ticket;  // blocks of the update kernel that have finished (0 between launches)
};
enum { ST_RUN = 0, ST_CONV = 1, ST_NOCONV = 2, ST_BREAK = 3, ST_UPDATE = 4 };

constexpr int kRedThreads = 256;

__device__ double sum_partials(const double* part, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  return block_sum(v, red);
}

// The same sum of partials that other blocks of the running kernel wrote
// (loads that bypass L1).
__device__ double sum_partials_cg(const double* part, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(part + i);
  return block_sum(v, red);
}

// The update and direction kernels read and write their vectors with 16-byte
// accesses (four floats or two doubles per thread and step); the solver's
// vectors start at multiples of 4 entries of one workspace, so every one of
// them is 16-byte aligned, and the last n % W entries run in a scalar tail.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int W = 4;
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int W = 2;
};

template <typename T>
__global__ void k_cg_init(int64_t n, const T* __restrict__ r, const T* __restrict__ dinv, T* __restrict__ z,
                          T* __restrict__ p, const T* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[32];
  using A = typename DotAcc<T>::type;
  A rz = 0, rr = 0, bb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = r[i];
    const T zi = ri * dinv[i];
    z[i] = zi;
    p[i] = zi;
    rz += (A)ri * (A)zi;
    rr += (A)ri * (A)ri;
    if (b) bb += (A)b[i] * (A)b[i];
  }
  double s;
  s = block_sum((double)rz, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  s = block_sum((double)rr, red);
  if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = s;
  s = block_sum((double)bb, red);
  if (threadIdx.x == 0) part[2 * gridDim.x + blockIdx.x] = s;
}

// bb_given >= 0: use it as ||b||^2 (inner solves of the refinement use a
// normalised right-hand side), else sum the b partials.
__global__ void k_cg_init_scalars(CgScalars* sc, const double* __restrict__ part, int nb, double rtol,
                                  double bb_given, int maxit) {
  __shared__ double red[32];
  const double rz = sum_partials(part, nb, red);
  const double rr = sum_partials(part + nb, nb, red);
  const double bb = sum_partials(part + 2 * nb, nb, red);
  if (threadIdx.x == 0) {
    sc->rzb[0] = rz;
    sc->rr = rr;
    sc->bb = bb_given >= 0 ? bb_given : bb;
    sc->tol2 = rtol * rtol * sc->bb;
    sc->it = 0;
    sc->it1 = 0;
    sc->maxit = maxit;
    sc->status = ST_RUN;
    sc->done = 0;
    sc->ru = 0;
    sc->upd2 = 0.0;
    sc->ticket = 0;
    if (rr <= sc->tol2) {
      sc->done = 1;
      sc->status = ST_CONV;
    }
    if (!isfinite(rz) || !isfinite(rr)) {
      sc->done = 1;
      sc->status = ST_BREAK;
    }
  }
}

// x += a p, r -= a q, z = r dinv with a = (r.z) / (p.q), the p.q partials
// (pq_part, written by the scatter) summed by every block; partials of r.z
// and r.r to part_out[0, nb) and part_out[nb, 2 nb). A non-positive or
// non-finite p.q stops the solve (breakdown) in every block alike. The last
// block to finish (an atomic ticket: no block waits for another) sums the
// r.z and r.r partials in the fixed order and takes the iteration's
// decisions (convergence test, beta, the next r.z slot) for the direction
// kernel.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_cg_update(int64_t n, CgScalars* __restrict__ sc, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
            const T* __restrict__ p, const T* __restrict__ q, const T* __restrict__ dinv,
            const double* __restrict__ pq_part, double* __restrict__ part_out, int nb) {
  __shared__ double red[32];
  __shared__ double s_alpha;
  __shared__ int s_ok;
  if (sc->done) return;
  const double pq = sum_partials(pq_part, nb, red);
  if (threadIdx.x == 0) {
    const int it = sc->it;
    const bool ok = pq > 0.0 && isfinite(pq);
    s_ok = ok;
    s_alpha = ok ? sc->rzb[it & 1] / pq : 0.0;
    if (blockIdx.x == 0) {
      if (ok) {
        sc->it1 = it + 1;
      } else {
        sc->done = 1;
        sc->status = ST_BREAK;
      }
    }
  }
  __syncthreads();
  if (!s_ok) return;
  const T a = (T)s_alpha;
  using A = typename DotAcc<T>::type;
  using V = typename Vec16<T>::V;
  constexpr int W = Vec16<T>::W;
  A rz = 0, rr = 0;
  const int64_t nv = n / W, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t j = tid; j < nv; j += stride) {
    V xv = reinterpret_cast<const V*>(x)[j], rv = reinterpret_cast<const V*>(r)[j];
    const V pv = reinterpret_cast<const V*>(p)[j], qv = reinterpret_cast<const V*>(q)[j];
    const V dv = reinterpret_cast<const V*>(dinv)[j];
    V zv;
    T* xs = reinterpret_cast<T*>(&xv);
    T* rs = reinterpret_cast<T*>(&rv);
    T* zs = reinterpret_cast<T*>(&zv);
    const T* ps = reinterpret_cast<const T*>(&pv);
    const T* qs = reinterpret_cast<const T*>(&qv);
    const T* ds = reinterpret_cast<const T*>(&dv);
#pragma unroll
    for (int u = 0; u < W; ++u) {
      xs[u] += a * ps[u];
      const T ri = rs[u] - a * qs[u];
      rs[u] = ri;
      const T zi = ri * ds[u];
      zs[u] = zi;
      rz += (A)ri * (A)zi;
      rr += (A)ri * (A)ri;
    }
    reinterpret_cast<V*>(x)[j] = xv;
    reinterpret_cast<V*>(r)[j] = rv;
    reinterpret_cast<V*>(z)[j] = zv;
  }
  for (int64_t i = nv * W + tid; i < n; i += stride) {
    x[i] += a * p[i];
    const T ri = r[i] - a * q[i];
    r[i] = ri;
    const T zi = ri * dinv[i];
    z[i] = zi;
    rz += (A)ri * (A)zi;
    rr += (A)ri * (A)ri;
  }
  double s = block_sum((double)rz, red);
  if (threadIdx.x == 0) part_out[blockIdx.x] = s;
  s = block_sum((double)rr, red);
  if (threadIdx.x == 0) part_out[gridDim.x + blockIdx.x] = s;
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const double rzt = sum_partials_cg(part_out, gridDim.x, red);
  const double rrt = sum_partials_cg(part_out + gridDim.x, gridDim.x, red);
  if (threadIdx.x == 0) {
    sc->ticket = 0;
    const int it = sc->it1;
    int status = ST_RUN;
    if (!isfinite(rzt) || !isfinite(rrt)) {
      status = ST_BREAK;
    } else if (sc->ru && (rrt <= sc->upd2 || rrt <= sc->tol2)) {
      // reliable-update mode: hand over to the host for an FP64 update (the
      // true residual decides convergence); beta waits for the new residual
      status = ST_UPDATE;
    } else if (rrt <= sc->tol2) {
      status = ST_CONV;
    } else if (it >= sc->maxit) {
      status = ST_NOCONV;
    }
    sc->it = it;
    sc->rr = rrt;
    if (status == ST_RUN) {
      sc->beta = rzt / sc->rzb[(it - 1) & 1];
      sc->rzb[it & 1] = rzt;
    } else {
      sc->status = status;
      sc->done = 1;
      if (status == ST_UPDATE) sc->rz_new = rzt;
    }
  }
}

// The next search direction p = z + beta p, with beta and the decision to go
// on taken by the update kernel's last block.
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_cg_direction(int64_t n, const CgScalars* __restrict__ sc, const T* __restrict__ z, T* __restrict__ p) {
  if (sc->done) return;
  const T b = (T)sc->beta;
  using V = typename Vec16<T>::V;
  constexpr int W = Vec16<T>::W;
  const int64_t nv = n / W, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t j = tid; j < nv; j += stride) {
    const V zv = reinterpret_cast<const V*>(z)[j];
    V pv = reinterpret_cast<const V*>(p)[j];
    const T* zs = reinterpret_cast<const T*>(&zv);
    T* ps = reinterpret_cast<T*>(&pv);
#pragma unroll
    for (int u = 0; u < W; ++u) ps[u] = zs[u] + b * ps[u];
    reinterpret_cast<V*>(p)[j] = pv;
  }
  for (int64_t i = nv * W + tid; i < n; i += stride) p[i] = z[i] + b * p[i];
}

// After a reliable update replaced r: z = r dinv and partials of r.z.
template <typename T>
__global__ void k_cg_rz(int64_t n, const T* __restrict__ r, const T* __restrict__ dinv, T* __restrict__ z,
                        double* __restrict__ part) {
  __shared__ double red[32];
  using A = typename DotAcc<T>::type;
  A rz = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = r[i];
    const T zi = ri * dinv[i];
    z[i] = zi;
    rz += (A)ri * (A)zi;
  }
  const double s = block_sum((double)rz, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Resume after a reliable update: beta from the new r.z, next update
// threshold, iteration continues (p = z + beta p follows).
__global__ void k_cg_resume(CgScalars* sc, const double* __restrict__ part, int nb, double upd2) {
  __shared__ double red[32];
  const double rz = sum_partials(part, nb, red);
  if (threadIdx.x == 0) {
    // the stopped iteration advanced `it` but kept its old r.z in slot it - 1
    const int it = sc->it;
    sc->beta = rz / sc->rzb[(it - 1) & 1];
    sc->rzb[it & 1] = rz;
    sc->upd2 = upd2;
    sc->status = ST_RUN;
    sc->done = 0;
    sc->ticket = 0;
    if (!isfinite(rz) || !(rz > 0.0)) {
      sc->done = 1;
      sc->status = ST_BREAK;
    }
  }
}

__global__ void k_cg_set_ru(CgScalars* sc, double upd2) {
  sc->ru = 1;
  sc->upd2 = upd2;
}

// x += (double) d; d = 0 (fold the FP32 increment into the FP64 solution).
__global__ void k_fold(int64_t n, double* __restrict__ x, float* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += (double)d[i];
    d[i] = 0.0f;
  }
}

__global__ void k_cast_r32(int64_t n, const double* __restrict__ r, float* __restrict__ r32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r32[i] = (float)r[i];
}

template <typename T>
__global__ void k_cg_p(int64_t n, const CgScalars* __restrict__ sc, const T* __restrict__ z, T* __restrict__ p) {
  if (sc->done) return;
  const T b = (T)sc->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + b * p[i];
}

// r = b - y, and partials of r.r (FP64 true residual).
template <typename TB>
__global__ void k_residual(int64_t n, const TB* __restrict__ b, const double* __restrict__ y, double* __restrict__ r,
                           double* __restrict__ part) {
  __shared__ double red[32];
  double rr = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = (double)b[i] - y[i];
    r[i] = ri;
    rr += ri * ri;
  }
  const double s = block_sum(rr, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sumsq(int64_t n, const double* __restrict__ v, double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += v[i] * v[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_to(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double red[32];
  const double s = sum_partials(part, nb, red);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_scale_to_f32(int64_t n, const double* __restrict__ r, const double* __restrict__ rr,
                               float* __restrict__ r32, float* __restrict__ x32) {
  const double inv = 1.0 / sqrt(*rr);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    r32[i] = (float)(r[i] * inv);
    x32[i] = 0.0f;
  }
}

__global__ void k_axpy_scaled(int64_t n, const double* __restrict__ rr, const float* __restrict__ d,
                              double* __restrict__ x) {
  const double s = sqrt(*rr);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += s * (double)d[i];
}

// a = 1 / a in place (the Jacobi preconditioner's reciprocal diagonal, once
// per solve, so that every iteration multiplies: an FP64 division is a
// multi-instruction sequence on GB300's FP64 pipe, and the FP64 vector
// update was bound by it rather than by HBM).
__global__ void k_recip(int64_t n, double* __restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = 1.0 / a[i];
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

__global__ void k_cast_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Workspace carved out of the form's buffers.
struct Work {
  int64_t n;
  int nb;                         // blocks of the vector kernels (and partials)
  double *x, *r, *z, *p, *q, *diag, *t;  // FP64 vectors (diag: the reciprocal Jacobi diagonal)
  float *x32, *r32, *z32, *p32, *q32, *diag32;
  double* part;                   // 3 * nb partials
  double* scal;                   // misc scalars (rr of refinement)
  CgScalars* sc;
};

fem_status get_work(fem_form* f, bool mixed, Work& w) {
  const int64_t n = fem_form_len(f);
  const int64_t np = (n + 3) & ~(int64_t)3;  // vector stride: every vector 16-byte aligned
  w.n = n;
  w.nb = fem_scatter_blocks(n);
  const size_t need64 = (size_t)7 * np;
  if (f->work64_len < need64) {
    dev_free(f->d_work64);
    FEM_TRY(dev_alloc(&f->d_work64, need64));
    f->work64_len = need64;
  }
  double* b = f->d_work64;
  w.x = b; w.r = b + np; w.z = b + 2 * np; w.p = b + 3 * np; w.q = b + 4 * np; w.diag = b + 5 * np;
  w.t = b + 6 * np;
  if (mixed) {
    const size_t need32 = (size_t)6 * np;
    if (f->work32_len < need32) {
      dev_free(f->d_work32);
      FEM_TRY(dev_alloc(&f->d_work32, need32));
      f->work32_len = need32;
    }
    float* a = f->d_work32;
    w.x32 = a; w.r32 = a + np; w.z32 = a + 2 * np; w.p32 = a + 3 * np; w.q32 = a + 4 * np;
    w.diag32 = a + 5 * np;
  }
  const size_t red_need = (size_t)3 * w.nb + 16 + (sizeof(CgScalars) + 7) / 8;
  if (f->red_len < red_need) {
    dev_free(f->d_red);
    FEM_TRY(dev_alloc(&f->d_red, red_need));
    f->red_len = red_need;
  }
  w.part = f->d_red;
  w.scal = f->d_red + 3 * w.nb;
  w.sc = reinterpret_cast<CgScalars*>(f->d_red + 3 * w.nb + 16);
  return FEM_OK;
}

// One CG iteration on vectors of type T.
// dtype: element-kernel type (FEM_F64, FEM_F32 or FEM_DF64); the vectors are T.
template <typename T>
fem_status cg_iteration(const fem_form* f, const Work& w, int dtype, T* x, T* r, T* z, T* p, T* q, const T* dinv,
                        cudaStream_t s) {
  const int* skip = &w.sc->done;
  const int vt = std::is_same<T, float>::value ? FEM_F32 : FEM_F64;
  FEM_TRY(fem_launch_apply_element(f, dtype, p, f->d_ye, s, skip, true));
  FEM_TRY(fem_launch_scatter(f, vt, f->d_ye, q, f->d_ess_mask, p, w.part, w.nb, s, skip, true));
  k_cg_update<T><<<w.nb, kRedThreads, 0, s>>>(w.n, w.sc, x, r, z, p, q, dinv, w.part, w.part + w.nb, w.nb);
  k_cg_direction<T><<<w.nb, kRedThreads, 0, s>>>(w.n, w.sc, z, p);
  FEM_LAUNCHED();
  return FEM_OK;
}

// Run CG iterations until the device `done` word is set. With use_graph the
// check_every iterations are captured once into a graph on a private stream
// and replayed on `s`.
template <typename T>
fem_status cg_loop(fem_form* f, const Work& w, int dtype, T* x, T* r, T* z, T* p, T* q, const T* dinv,
                   const fem_solve_opts& o, cudaStream_t s, int* status_out, int* it_out) {
  const int k = o.check_every > 0 ? o.check_every : 16;
  cudaGraphExec_t exec = nullptr;
  if (o.use_graph) {
    cudaStream_t cs;
    FEM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    fem_status st = FEM_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = fem_fail(FEM_ECUDA, "solve: stream capture failed to begin");
    } else {
      for (int i = 0; i < k && st == FEM_OK; ++i) st = cg_iteration<T>(f, w, dtype, x, r, z, p, q, dinv, cs);
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (st == FEM_OK && e != cudaSuccess) st = fem_fail(FEM_ECUDA, "solve: end capture: %s", cudaGetErrorString(e));
    }
    if (st == FEM_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "solve: graph instantiation failed");
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st != FEM_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      return st;
    }
  }
  int* h = f->h_pinned;
  fem_status st = FEM_OK;
  const int max_rounds = o.maxit / k + 2;
  for (int round = 0; round < max_rounds; ++round) {
    if (exec) {
      if (cudaGraphLaunch(exec, s) != cudaSuccess) {
        st = fem_fail(FEM_ECUDA, "solve: graph launch failed");
        break;
      }
    } else {
      for (int i = 0; i < k && st == FEM_OK; ++i) st = cg_iteration<T>(f, w, dtype, x, r, z, p, q, dinv, s);
      if (st != FEM_OK) break;
    }
    if (cudaMemcpyAsync(h, &w.sc->it, 4 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = fem_fail(FEM_ECUDA, "solve: status read failed: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    if (h[1]) break;  // done
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (st != FEM_OK) return st;
  *it_out = h[0];
  *status_out = h[1] ? h[2] : ST_NOCONV;
  return FEM_OK;
}

// ||b - A_c x||^2 into *out (device), r = b - A_c x (FP64).
// r = b - A_c x and ||r||^2 (to *out), FP64 vectors; the operator in FP64
// or (arith FEM_DF64) in double-float, which gives the same residual to about
// 1e-13 relative at a quarter of the FP64 apply's time.
fem_status true_residual(fem_form* f, const Work& w, const double* b, const double* x, double* r, double* out,
                         cudaStream_t s, int arith = FEM_F64) {
  FEM_TRY(fem_launch_zero_ess(f, FEM_F64, x, w.t, s));
  FEM_TRY(fem_launch_apply_element(f, arith, w.t, f->d_ye, s, nullptr, true));
  FEM_TRY(fem_launch_scatter(f, FEM_F64, f->d_ye, w.q, f->d_ess_mask, x, nullptr, 0, s, nullptr, true));
  k_residual<double><<<w.nb, 256, 0, s>>>(w.n, b, w.q, r, w.part);
  k_sum_to<<<1, kRedThreads, 0, s>>>(w.part, w.nb, out);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status read_doubles(fem_form* f, const double* d, int n, double* h, cudaStream_t s) {
  FEM_CUDA(cudaMemcpyAsync(f->h_pinned + 8, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  std::memcpy(h, f->h_pinned + 8, sizeof(double) * n);
  return FEM_OK;
}

}  // namespace

__global__ void k_dot_partials(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                               double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

extern "C" fem_status fem_compliance(const fem_form* fc, const double* b, const double* u, double* J, void* stream) {
  if (!fc || !b || !u || !J) return fem_fail(FEM_EINVAL, "fem_compliance: NULL argument");
  fem_form* f = const_cast<fem_form*>(fc);
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  FEM_TRY(get_work(f, false, w));
  k_dot_partials<<<w.nb, 256, 0, s>>>(w.n, b, u, w.part);
  k_sum_to<<<1, kRedThreads, 0, s>>>(w.part, w.nb, J);
  FEM_LAUNCHED();
  return FEM_OK;
}

// inner_rtol <= 0 selects the default of the mode, measured on the
// ~2e7-DOF p = 4 and p = 6 diffusion problems (lognormal kappa, perturbed
// hexes) and the p = 2, 8 ones of ~4e6 DOFs: restarted FP32 inner CG 1e-4
// (with the last pass stopping at half the tolerance; p = 4 1.53 s against
// 1.67 s at 1e-3), reliable updates 0.1 (1e-2: 2.30 -> 1.44 s at p = 4,
// 2.78 -> 1.35 s at p = 6), the multigrid FP32 outer operator 3e-4, the
// batched mixed solve 1e-4 (1e-3 was slower there).
double fem_inner_rtol(const fem_solve_opts& o, int which) {
  if (o.inner_rtol > 0) return o.inner_rtol;
  switch (which) {
    case 1: return 3e-4;   // fem_mg_solve, FP32 outer operator
    case 2: return 1e-4;   // fem_batch_solve
    default: return o.precision == FEM_SOLVE_MIXED_RU ? 0.1 : 1e-4;
  }
}

extern "C" void fem_solve_opts_default(fem_solve_opts* o) {
  if (!o) return;
  o->rtol = 1e-10;
  o->maxit = 20000;
  o->precision = FEM_SOLVE_F64;
  o->inner_rtol = 0.0;  // the mode's measured default (fem_inner_rtol)
  o->max_outer = 30;
  o->check_every = 16;
  o->use_graph = 1;
  o->precond = FEM_PC_JACOBI;
}

extern "C" fem_status fem_solve(const fem_form* fc, const double* b, double* xio, const fem_solve_opts* opts,
                                fem_solve_info* info, void* stream) {
  if (!fc || !b || !xio) return fem_fail(FEM_EINVAL, "fem_solve: NULL argument");
  if (!fc->d_ess_mask) return fem_fail(FEM_EINVAL, "fem_solve: call fem_form_set_essential first (n may be 0)");
  if (fc->kind == FEM_CONVECTION) return fem_fail(FEM_EINVAL, "fem_solve: CG needs a symmetric (mass or diffusion) form");
  fem_solve_opts o;
  fem_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0) || o.maxit <= 0) return fem_fail(FEM_EINVAL, "fem_solve: rtol > 0 and maxit > 0 required");
  o.inner_rtol = fem_inner_rtol(o, 0);
  if (o.precision != FEM_SOLVE_F64 && o.precision != FEM_SOLVE_MIXED && o.precision != FEM_SOLVE_DF64 &&
      o.precision != FEM_SOLVE_MIXED_RU)
    return fem_fail(FEM_EINVAL, "fem_solve: unknown precision %d", o.precision);
  if (o.precond != FEM_PC_JACOBI && o.precond != FEM_PC_NONE)
    return fem_fail(FEM_EINVAL, "fem_solve: unknown preconditioner %d", o.precond);
  fem_form* f = const_cast<fem_form*>(fc);
  cudaStream_t s = (cudaStream_t)stream;
  const bool ru = o.precision == FEM_SOLVE_MIXED_RU;
  const bool mixed = o.precision == FEM_SOLVE_MIXED || ru;
  Work w;
  FEM_TRY(get_work(f, mixed, w));
  if (mixed) FEM_TRY(fem_form_ensure_f32(f, s));
  const int op64 = o.precision == FEM_SOLVE_DF64 ? FEM_DF64 : FEM_F64;  // FP64-vector operator
  if (op64 == FEM_DF64) FEM_TRY(fem_form_ensure_df64(f, s));
  const int64_t n = w.n;
  FEM_CUDA(cudaMemcpyAsync(w.x, xio, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (o.precond == FEM_PC_NONE) {
    k_fill<<<w.nb, 256, 0, s>>>(n, 1.0, w.diag);
    FEM_LAUNCHED();
  } else {
    FEM_TRY(fem_assemble_diagonal(f, w.diag, 1, s));
    k_recip<<<w.nb, 256, 0, s>>>(n, w.diag);  // w.diag holds the reciprocal from here on
    FEM_LAUNCHED();
  }
  fem_solve_info inf;
  std::memset(&inf, 0, sizeof inf);
  double hb[2];
  int total_it = 0, outer = 0, status = ST_NOCONV;
  double* rr_dev = w.scal;       // ||r||^2 of the last true residual
  // ||b||^2
  k_sumsq<<<w.nb, 256, 0, s>>>(n, b, w.part);
  k_sum_to<<<1, kRedThreads, 0, s>>>(w.part, w.nb, w.scal + 1);
  FEM_LAUNCHED();
  FEM_TRY(read_doubles(f, w.scal + 1, 1, hb, s));
  const double bb = hb[0];
  inf.bnorm = std::sqrt(bb);
  const double tol2 = o.rtol * o.rtol * bb;
  if (!std::isfinite(bb)) {
    if (info) *info = inf;
    return fem_fail(FEM_EBREAKDOWN, "fem_solve: non-finite right-hand side");
  }
  if (!(bb > 0)) {
    // b = 0: the solution of A_c x = 0 is x = 0
    FEM_CUDA(cudaMemsetAsync(xio, 0, sizeof(double) * n, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    inf.converged = 1;
    if (info) *info = inf;
    return FEM_OK;
  }
  double rr = 0;
  // The reliable updates compute their residuals with the double-float
  // operator while the previous residual is above 1e-6 relative (its
  // rounding, at most ~1e-11 relative to b on the coefficient fields tested,
  // is then far below what the next FP32 segment resolves), with the FP64
  // operator after that; a residual that meets the tolerance is always
  // recomputed in FP64, which alone decides convergence (and gives relres).
  // (The restarted refinement keeps FP64 residuals: the same change there
  // moved its pass boundary, 4 -> 5 passes and 1.68 -> 2.05 s at p = 4.)
  if (ru) FEM_TRY(fem_form_ensure_df64(f, s));
  double prev_rel2 = 1.0;
  auto residual = [&](double& out) -> fem_status {
    const int arith = (ru && prev_rel2 > 1e-12) ? FEM_DF64 : FEM_F64;
    FEM_TRY(true_residual(f, w, b, w.x, w.r, rr_dev, s, arith));
    FEM_TRY(read_doubles(f, rr_dev, 1, &out, s));
    if (arith != FEM_F64 && std::isfinite(out) && out <= tol2) {
      FEM_TRY(true_residual(f, w, b, w.x, w.r, rr_dev, s));
      FEM_TRY(read_doubles(f, rr_dev, 1, &out, s));
    }
    prev_rel2 = out / bb;
    return FEM_OK;
  };
  if (ru) {
    // FP32 CG with reliable updates: the search direction is never restarted;
    // when the FP32 residual has dropped by delta since the last update, the
    // FP32 increment is folded into the FP64 solution and the residual is
    // replaced by the FP64 true residual b - A_c x.
    const double delta2 = o.inner_rtol * o.inner_rtol;
    float* x32 = w.x32;
    float* r32 = w.r32;
    FEM_TRY(residual(rr));
    status = ST_NOCONV;
    if (!std::isfinite(rr)) status = ST_BREAK;
    else if (rr <= tol2) status = ST_CONV;
    if (status == ST_NOCONV) {
      k_cast_f32<<<w.nb, 256, 0, s>>>(n, w.diag, w.diag32);
      k_cast_r32<<<w.nb, 256, 0, s>>>(n, w.r, r32);
      FEM_CUDA(cudaMemsetAsync(x32, 0, sizeof(float) * n, s));
      k_cg_init<float><<<w.nb, 256, 0, s>>>(n, r32, w.diag32, w.z32, w.p32, nullptr, w.part);
      k_cg_init_scalars<<<1, kRedThreads, 0, s>>>(w.sc, w.part, w.nb, o.rtol, bb, o.maxit);
      k_cg_set_ru<<<1, 1, 0, s>>>(w.sc, delta2 * rr);
      FEM_LAUNCHED();
      for (;;) {
        fem_solve_opts oi = o;
        int st_in = ST_NOCONV, it_in = 0;
        FEM_TRY(cg_loop<float>(f, w, FEM_F32, x32, r32, w.z32, w.p32, w.q32, w.diag32, oi, s, &st_in, &it_in));
        total_it = it_in;  // the device counter runs across updates
        k_fold<<<w.nb, 256, 0, s>>>(n, w.x, x32);
        FEM_LAUNCHED();
        ++outer;
        FEM_TRY(residual(rr));
        if (!std::isfinite(rr) || st_in == ST_BREAK) {
          status = ST_BREAK;
          break;
        }
        if (rr <= tol2) {
          status = ST_CONV;
          break;
        }
        if (total_it >= o.maxit || st_in == ST_NOCONV || outer > 100000) {
          status = ST_NOCONV;
          break;
        }
        k_cast_r32<<<w.nb, 256, 0, s>>>(n, w.r, r32);
        k_cg_rz<float><<<w.nb, 256, 0, s>>>(n, r32, w.diag32, w.z32, w.part);
        k_cg_resume<<<1, kRedThreads, 0, s>>>(w.sc, w.part, w.nb, delta2 * rr);
        k_cg_p<float><<<w.nb, 256, 0, s>>>(n, w.sc, w.z32, w.p32);
        FEM_LAUNCHED();
      }
    }
  }
  for (; !ru;) {
    FEM_TRY(residual(rr));
    if (!std::isfinite(rr)) {
      status = ST_BREAK;
      break;
    }
    if (rr <= tol2) {
      status = ST_CONV;
      break;
    }
    if (total_it >= o.maxit || (mixed && outer >= o.max_outer) || (!mixed && outer > o.max_outer)) {
      status = ST_NOCONV;
      break;
    }
    int st_in = ST_NOCONV, it_in = 0;
    fem_solve_opts oi = o;
    oi.maxit = o.maxit - total_it;
    if (!mixed) {
      // restart CG from the current x with the true residual
      k_cg_init<double><<<w.nb, 256, 0, s>>>(n, w.r, w.diag, w.z, w.p, nullptr, w.part);
      k_cg_init_scalars<<<1, kRedThreads, 0, s>>>(w.sc, w.part, w.nb, o.rtol, bb, oi.maxit);
      FEM_LAUNCHED();
      FEM_TRY(cg_loop<double>(f, w, op64, w.x, w.r, w.z, w.p, w.q, w.diag, oi, s, &st_in, &it_in));
    } else {
      // inner FP32 solve of A d = r / ||r|| to inner_rtol, then x += ||r|| d;
      // a pass that needs less than that to reach the tolerance stops at half
      // of the tolerance (rtol ||b|| / 2) instead of a full inner_rtol drop
      const double inner = std::max(o.inner_rtol, 0.5 * std::sqrt(tol2 / rr));
      k_cast_f32<<<w.nb, 256, 0, s>>>(n, w.diag, w.diag32);
      k_scale_to_f32<<<w.nb, 256, 0, s>>>(n, w.r, rr_dev, w.r32, w.x32);
      k_cg_init<float><<<w.nb, 256, 0, s>>>(n, w.r32, w.diag32, w.z32, w.p32, nullptr, w.part);
      k_cg_init_scalars<<<1, kRedThreads, 0, s>>>(w.sc, w.part, w.nb, inner, 1.0, oi.maxit);
      FEM_LAUNCHED();
      FEM_TRY(cg_loop<float>(f, w, FEM_F32, w.x32, w.r32, w.z32, w.p32, w.q32, w.diag32, oi, s, &st_in, &it_in));
      k_axpy_scaled<<<w.nb, 256, 0, s>>>(n, rr_dev, w.x32, w.x);
      FEM_LAUNCHED();
    }
    total_it += it_in;
    outer += 1;
    if (st_in == ST_BREAK) {
      status = ST_BREAK;
      break;
    }
  }
  FEM_CUDA(cudaMemcpyAsync(xio, w.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  inf.iterations = total_it;
  inf.outer = outer;
  inf.relres = std::sqrt(rr / bb);
  inf.converged = status == ST_CONV;
  if (info) *info = inf;
  if (status == ST_BREAK) return fem_fail(FEM_EBREAKDOWN, "fem_solve: CG breakdown (p^T A p <= 0 or non-finite)");
  if (status != ST_CONV)
    return fem_fail(FEM_ENOCONV, "fem_solve: no convergence after %d iterations (relres %.3e)", total_it,
                    inf.relres);
  return FEM_OK;
}
