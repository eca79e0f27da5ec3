// Device side of the sharded operator (the plan is built in fem_shard.cpp):
// the halo sum that turns a rank's partial L-vector into the assembled one
// (the paper's P^T and P, Sec. 4.3, done in one exchange round), owned-DOF
// dot products with an all-reduce, and Jacobi-PCG on the sharded operator
// (Sec. 5.2's CGSolver iteration, with the parallel inner products a
// distributed run needs).
//
// Halo sum: pack the partials of every exchange slot into the send buffer,
// let the caller's transport swap send and receive buffers with the
// neighbours, then for each DOF held by several ranks add the partials of
// all holders in ascending rank order (this rank's own value at its place
// in that order). Every holder adds the same numbers in the same order, so
// the assembled values agree bit for bit across ranks.
#include <cmath>
#include <cstring>

#include "fem_internal.h"
#include "k_common.cuh"

namespace {

constexpr int kT = 256;

// send[base(t) + c * cnt(t)] = y[c * ndof + slot_dof[t]], where slot t
// belongs to neighbour k = slot_nbr[t], base(t) = vdim * slot_off[k] +
// (t - slot_off[k]) and cnt(t) = slot_off[k + 1] - slot_off[k].
__global__ void k_sh_pack(int64_t nslots, int vdim, int64_t ndof, const int32_t* __restrict__ slot_dof,
                          const int32_t* __restrict__ slot_nbr, const int64_t* __restrict__ slot_off,
                          const double* __restrict__ y, double* __restrict__ send) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nslots; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = slot_nbr[t];
    const int64_t o = slot_off[k], cnt = slot_off[k + 1] - o;
    const int64_t base = vdim * o + (t - o);
    const int32_t i = slot_dof[t];
    for (int c = 0; c < vdim; ++c) send[base + c * cnt] = y[c * ndof + i];
  }
}

// y[c * ndof + comb_dof[j]] = sum over the entries of j, in order, of the
// own partial (src < 0) or the partial received in slot src.
__global__ void k_sh_combine(int64_t nshared, int vdim, int64_t ndof, const int32_t* __restrict__ comb_dof,
                             const int32_t* __restrict__ comb_off, const int32_t* __restrict__ comb_src,
                             const int32_t* __restrict__ slot_nbr, const int64_t* __restrict__ slot_off,
                             const double* __restrict__ recv, double* __restrict__ y) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nshared;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = comb_dof[j];
    const int32_t a = comb_off[j], b = comb_off[j + 1];
    for (int c = 0; c < vdim; ++c) {
      const double own = y[c * ndof + i];
      double v = 0.0;
      for (int32_t t = a; t < b; ++t) {
        const int32_t src = comb_src[t];
        if (src < 0) {
          v += own;
        } else {
          const int k = slot_nbr[src];
          const int64_t o = slot_off[k], cnt = slot_off[k + 1] - o;
          v += recv[vdim * o + (src - o) + c * cnt];
        }
      }
      y[c * ndof + i] = v;
    }
  }
}

// Per-block partial sums of a . b over owned entries (entry c * ndof + i is
// owned when DOF i is); two products at once when a2 != nullptr.
__global__ void k_sh_dot(int64_t n, int64_t ndof, const uint8_t* __restrict__ owned, const double* __restrict__ a,
                         const double* __restrict__ b, const double* __restrict__ a2,
                         const double* __restrict__ b2, double* __restrict__ part) {
  __shared__ double red[32];
  double s1 = 0.0, s2 = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    if (!owned[e % ndof]) continue;
    s1 += a[e] * b[e];
    if (a2) s2 += a2[e] * b2[e];
  }
  double t = block_sum(s1, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (a2) {
    t = block_sum(s2, red);
    if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t;
  }
}

// out[m] = sum of part[m * nb, (m + 1) * nb), fixed order (one block).
__global__ void k_sh_sum(const double* __restrict__ part, int nb, int m, double* __restrict__ out) {
  __shared__ double red[32];
  for (int j = 0; j < m; ++j) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[j * nb + i];
    v = block_sum(v, red);
    if (threadIdx.x == 0) out[j] = v;
  }
}

__global__ void k_sh_to_local(int64_t nl, int vdim, int64_t ndof_g, const int64_t* __restrict__ l2g,
                              const double* __restrict__ xg, double* __restrict__ xl) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < vdim; ++c) xl[c * nl + i] = xg[c * ndof_g + l2g[i]];
}

__global__ void k_sh_to_global(int64_t nl, int vdim, int64_t ndof_g, const int64_t* __restrict__ l2g,
                               const uint8_t* __restrict__ owned, const double* __restrict__ xl,
                               double* __restrict__ xg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl; i += (int64_t)gridDim.x * blockDim.x)
    if (owned[i])
      for (int c = 0; c < vdim; ++c) xg[c * ndof_g + l2g[i]] = xl[c * nl + i];
}

__global__ void k_sh_zero_ess(int64_t n, const uint8_t* __restrict__ mask, const double* __restrict__ x,
                              double* __restrict__ xz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    xz[i] = mask[i] ? 0.0 : x[i];
}

// y_i = v_i (or the constant c when v == nullptr) on essential entries.
__global__ void k_sh_ess_rows(int64_t n, const uint8_t* __restrict__ mask, const double* __restrict__ v, double c,
                              double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (mask[i]) y[i] = v ? v[i] : c;
}

// ---------------------------------------------------------------- PCG ----
// Scalars (device): S[0] = p.q, S[1] = r.z (new), S[2] = r.r, S[3 + (it & 1)]
// = r.z of iteration it; all-reduced sums where they are global.
__global__ void k_sh_cg_start(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                              const double* __restrict__ dinv, double* __restrict__ r, double* __restrict__ z,
                              double* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - q[i];
    const double zi = ri * dinv[i];
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
  }
}

__global__ void k_sh_copy_scalar(double* __restrict__ dst, const double* __restrict__ src) { *dst = *src; }

__global__ void k_sh_recip(int64_t n, double* __restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = 1.0 / a[i];
}

// x += a p, r -= a q, z = r dinv with a = S[3 + par] / S[0].
__global__ void k_sh_cg_update(int64_t n, const double* __restrict__ S, int par, double* __restrict__ x,
                               double* __restrict__ r, double* __restrict__ z, const double* __restrict__ p,
                               const double* __restrict__ q, const double* __restrict__ dinv) {
  const double a = S[3 + par] / S[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    const double ri = r[i] - a * q[i];
    r[i] = ri;
    z[i] = ri * dinv[i];
  }
}

// p = z + beta p with beta = S[1] / S[3 + par]; block 0 stores S[1] as the
// r.z of the next iteration (slot 3 + (1 - par), which no block reads here).
__global__ void k_sh_cg_direction(int64_t n, double* __restrict__ S, int par, const double* __restrict__ z,
                                  double* __restrict__ p) {
  const double rz = S[1];
  const double beta = rz / S[3 + par];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) S[3 + (1 - par)] = rz;
}

__global__ void k_sh_fill(int64_t n, double v, double* __restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

__global__ void k_sh_residual(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                              double* __restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - q[i];
}

// ------------------------------------------------------------- helpers ----
fem_status check_form(const fem_shard* sh, const fem_form* f, const char* who) {
  if (!sh || !f) return fem_fail(FEM_EINVAL, "%s: NULL argument", who);
  if (f->space != sh->lspace) return fem_fail(FEM_EINVAL, "%s: the form is not built on the shard's space", who);
  if (f->kind == FEM_CONVECTION) return fem_fail(FEM_EUNSUPPORTED, "%s: convection forms are not sharded", who);
  return FEM_OK;
}

fem_status sync_if(const fem_comm* comm, cudaStream_t s) {
  if (comm && comm->host_sync) FEM_CUDA(cudaStreamSynchronize(s));
  return FEM_OK;
}

// Partial L-vector y (this rank's elements only) -> assembled, consistent y.
fem_status halo_sum(const fem_shard* sh, int vdim, double* y, const fem_comm* comm, cudaStream_t s) {
  const int nn = (int)sh->nbr.size();
  if (nn == 0) return FEM_OK;
  if (!comm || !comm->exchange)
    return fem_fail(FEM_EINVAL, "shard: this rank has %d neighbours but no exchange callback", nn);
  const int64_t nslots = (int64_t)sh->slot_dof.size(), ndof = sh->lspace->ndof;
  k_sh_pack<<<grid_for(nslots, kT), kT, 0, s>>>(nslots, vdim, ndof, sh->d_slot_dof, sh->d_slot_nbr, sh->d_slot_off,
                                                 y, sh->d_send);
  FEM_LAUNCHED();
  FEM_TRY(sync_if(comm, s));
  const std::vector<int64_t>& off = vdim == 3 ? sh->xoff3 : sh->xoff1;
  if (comm->exchange(comm->ctx, nn, sh->nbr.data(), off.data(), sh->d_send, sh->d_recv, (void*)s) != 0)
    return fem_fail(FEM_ECUDA, "shard: the exchange callback failed");
  const int64_t nsh = (int64_t)sh->comb_dof.size();
  k_sh_combine<<<grid_for(nsh, kT), kT, 0, s>>>(nsh, vdim, ndof, sh->d_comb_dof, sh->d_comb_off, sh->d_comb_src,
                                                 sh->d_slot_nbr, sh->d_slot_off, sh->d_recv, y);
  FEM_LAUNCHED();
  return FEM_OK;
}

fem_status allreduce(const fem_comm* comm, double* vals, int n, cudaStream_t s) {
  if (!comm || !comm->allreduce) return FEM_OK;  // one rank: the local sum is the global one
  FEM_TRY(sync_if(comm, s));
  if (comm->allreduce(comm->ctx, vals, n, (void*)s) != 0)
    return fem_fail(FEM_ECUDA, "shard: the all-reduce callback failed");
  return FEM_OK;
}

fem_status ensure_red(const fem_shard* sh, int nb) {
  const size_t need = (size_t)2 * nb + 8;
  if (sh->red_len < need) {
    dev_free(sh->d_red);
    FEM_TRY(dev_alloc(&sh->d_red, need));
    sh->red_len = need;
  }
  if (!sh->h_pinned) FEM_CUDA(cudaMallocHost((void**)&sh->h_pinned, sizeof(double) * 8));
  return FEM_OK;
}

// Global owned dot products into S[0..m) (device), m = 1 or 2.
fem_status dots(const fem_shard* sh, int vdim, const double* a, const double* b, const double* a2,
                const double* b2, double* S, const fem_comm* comm, cudaStream_t s) {
  const int64_t ndof = sh->lspace->ndof, n = vdim * ndof;
  const int nb = grid_for(n, kT);
  FEM_TRY(ensure_red(sh, nb));
  const int m = a2 ? 2 : 1;
  k_sh_dot<<<nb, kT, 0, s>>>(n, ndof, sh->d_owned, a, b, a2, b2, sh->d_red);
  k_sh_sum<<<1, kT, 0, s>>>(sh->d_red, nb, m, S);
  FEM_LAUNCHED();
  return allreduce(comm, S, m, s);
}

fem_status apply_raw(const fem_shard* sh, const fem_form* f, const double* x, double* y, bool constrained,
                     double* xz, const fem_comm* comm, cudaStream_t s) {
  const int64_t n = fem_form_len(f);
  const double* xin = x;
  if (constrained) {
    k_sh_zero_ess<<<grid_for(n, kT), kT, 0, s>>>(n, f->d_ess_mask, x, xz);
    FEM_LAUNCHED();
    xin = xz;
  }
  FEM_TRY(fem_launch_apply_element(f, FEM_F64, xin, f->d_ye, s, nullptr, true));
  FEM_TRY(fem_launch_scatter(f, FEM_F64, f->d_ye, y, nullptr, nullptr, nullptr, 0, s, nullptr, true));
  FEM_TRY(halo_sum(sh, f->vdim, y, comm, s));
  if (constrained) {
    k_sh_ess_rows<<<grid_for(n, kT), kT, 0, s>>>(n, f->d_ess_mask, x, 0.0, y);
    FEM_LAUNCHED();
  }
  return FEM_OK;
}

fem_status ensure_work(const fem_shard* sh, size_t n) {
  if (sh->work_len < n) {
    dev_free(sh->d_work);
    FEM_TRY(dev_alloc(&sh->d_work, n));
    sh->work_len = n;
  }
  return FEM_OK;
}

fem_status read_scalars(const fem_shard* sh, const double* S, int n, double* h, cudaStream_t s) {
  FEM_CUDA(cudaMemcpyAsync(sh->h_pinned, S, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  std::memcpy(h, sh->h_pinned, sizeof(double) * n);
  return FEM_OK;
}

}  // namespace

extern "C" fem_status fem_shard_to_local(const fem_shard* sh, int vdim, const double* xg, double* xl,
                                         void* stream) {
  if (!sh || !xg || !xl || (vdim != 1 && vdim != 3)) return fem_fail(FEM_EINVAL, "fem_shard_to_local: arguments");
  const int64_t nl = sh->lspace->ndof;
  k_sh_to_local<<<grid_for(nl, kT), kT, 0, (cudaStream_t)stream>>>(nl, vdim, sh->ndof_global, sh->d_l2g, xg, xl);
  FEM_LAUNCHED();
  return FEM_OK;
}

extern "C" fem_status fem_shard_to_global(const fem_shard* sh, int vdim, const double* xl, double* xg,
                                          void* stream) {
  if (!sh || !xg || !xl || (vdim != 1 && vdim != 3)) return fem_fail(FEM_EINVAL, "fem_shard_to_global: arguments");
  const int64_t nl = sh->lspace->ndof;
  k_sh_to_global<<<grid_for(nl, kT), kT, 0, (cudaStream_t)stream>>>(nl, vdim, sh->ndof_global, sh->d_l2g,
                                                                     sh->d_owned, xl, xg);
  FEM_LAUNCHED();
  return FEM_OK;
}

extern "C" fem_status fem_shard_apply(const fem_shard* sh, const fem_form* f, const double* x, double* y,
                                      int constrained, const fem_comm* comm, void* stream) {
  FEM_TRY(check_form(sh, f, "fem_shard_apply"));
  if (!x || !y || x == y) return fem_fail(FEM_EINVAL, "fem_shard_apply: x, y NULL or aliased");
  if (constrained && !f->d_ess_mask) return fem_fail(FEM_EINVAL, "fem_shard_apply: constrained apply needs essential DOFs");
  cudaStream_t s = (cudaStream_t)stream;
  double* xz = nullptr;
  if (constrained) {
    FEM_TRY(ensure_work(sh, (size_t)fem_form_len(f)));
    xz = sh->d_work;
  }
  return apply_raw(sh, f, x, y, constrained != 0, xz, comm, s);
}

extern "C" fem_status fem_shard_diagonal(const fem_shard* sh, const fem_form* f, double* diag, int constrained,
                                         const fem_comm* comm, void* stream) {
  FEM_TRY(check_form(sh, f, "fem_shard_diagonal"));
  if (!diag) return fem_fail(FEM_EINVAL, "fem_shard_diagonal: NULL diag");
  if (constrained && !f->d_ess_mask) return fem_fail(FEM_EINVAL, "fem_shard_diagonal: constrained needs essential DOFs");
  cudaStream_t s = (cudaStream_t)stream;
  FEM_TRY(fem_assemble_diagonal(f, diag, 0, s));
  FEM_TRY(halo_sum(sh, f->vdim, diag, comm, s));
  if (constrained) {
    const int64_t n = fem_form_len(f);
    k_sh_ess_rows<<<grid_for(n, kT), kT, 0, s>>>(n, f->d_ess_mask, nullptr, 1.0, diag);
    FEM_LAUNCHED();
  }
  return FEM_OK;
}

extern "C" fem_status fem_shard_rhs(const fem_shard* sh, const fem_form* f, const double* fq, double* b,
                                    const fem_comm* comm, void* stream) {
  FEM_TRY(check_form(sh, f, "fem_shard_rhs"));
  if (!fq || !b) return fem_fail(FEM_EINVAL, "fem_shard_rhs: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  FEM_TRY(fem_rhs(f, fq, b, s));
  return halo_sum(sh, f->vdim, b, comm, s);
}

extern "C" fem_status fem_shard_dot(const fem_shard* sh, int vdim, const double* a, const double* b,
                                    double* out_host, const fem_comm* comm, void* stream) {
  if (!sh || !a || !b || !out_host || (vdim != 1 && vdim != 3))
    return fem_fail(FEM_EINVAL, "fem_shard_dot: arguments");
  cudaStream_t s = (cudaStream_t)stream;
  FEM_TRY(ensure_red(sh, grid_for((int64_t)vdim * sh->lspace->ndof, kT)));
  double* S = sh->d_red + sh->red_len - 8;
  FEM_TRY(dots(sh, vdim, a, b, nullptr, nullptr, S, comm, s));
  return read_scalars(sh, S, 1, out_host, s);
}

extern "C" fem_status fem_shard_solve(const fem_shard* sh, const fem_form* f, const double* b, double* xio,
                                      const fem_solve_opts* opts, fem_solve_info* info, const fem_comm* comm,
                                      void* stream) {
  FEM_TRY(check_form(sh, f, "fem_shard_solve"));
  if (!b || !xio) return fem_fail(FEM_EINVAL, "fem_shard_solve: NULL argument");
  if (!f->d_ess_mask) return fem_fail(FEM_EINVAL, "fem_shard_solve: set the essential DOFs first (n may be 0)");
  fem_solve_opts o;
  fem_solve_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0) || o.maxit <= 0) return fem_fail(FEM_EINVAL, "fem_shard_solve: rtol > 0 and maxit > 0 required");
  if (o.precond != FEM_PC_JACOBI && o.precond != FEM_PC_NONE)
    return fem_fail(FEM_EINVAL, "fem_shard_solve: unknown preconditioner %d", o.precond);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = fem_form_len(f);
  FEM_TRY(ensure_work(sh, (size_t)7 * n));
  double* w = sh->d_work;
  double *xz = w, *x = w + n, *r = w + 2 * n, *z = w + 3 * n, *p = w + 4 * n, *q = w + 5 * n, *diag = w + 6 * n;
  FEM_TRY(ensure_red(sh, grid_for(n, kT)));
  double* S = sh->d_red + sh->red_len - 8;
  FEM_CUDA(cudaMemcpyAsync(x, xio, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if (o.precond == FEM_PC_NONE) {
    k_sh_fill<<<grid_for(n, kT), kT, 0, s>>>(n, 1.0, diag);
    FEM_LAUNCHED();
  } else {
    FEM_TRY(fem_shard_diagonal(sh, f, diag, 1, comm, s));
    // the reciprocal diagonal: every iteration multiplies instead of dividing
    k_sh_recip<<<grid_for(n, kT), kT, 0, s>>>(n, diag);
    FEM_LAUNCHED();
  }
  fem_solve_info inf;
  std::memset(&inf, 0, sizeof inf);
  double h[3];
  FEM_TRY(dots(sh, f->vdim, b, b, nullptr, nullptr, S, comm, s));
  FEM_TRY(read_scalars(sh, S, 1, h, s));
  const double bb = h[0];
  inf.bnorm = std::sqrt(bb);
  if (!std::isfinite(bb)) return fem_fail(FEM_EBREAKDOWN, "fem_shard_solve: non-finite right-hand side");
  if (!(bb > 0)) {
    FEM_CUDA(cudaMemsetAsync(xio, 0, sizeof(double) * n, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    inf.converged = 1;
    if (info) *info = inf;
    return FEM_OK;
  }
  const double tol2 = o.rtol * o.rtol * bb;
  enum { RUN, CONV, NOCONV, BREAK } status = NOCONV;
  int total = 0, outer = 0;
  double rr = 0;
  const int gv = grid_for(n, kT);
  for (;;) {
    // true residual r = b - A_c x (restart point of every pass)
    FEM_TRY(apply_raw(sh, f, x, q, true, xz, comm, s));
    k_sh_residual<<<gv, kT, 0, s>>>(n, b, q, r);
    FEM_LAUNCHED();
    FEM_TRY(dots(sh, f->vdim, r, r, nullptr, nullptr, S + 2, comm, s));
    FEM_TRY(read_scalars(sh, S + 2, 1, &rr, s));
    if (!std::isfinite(rr)) {
      status = BREAK;
      break;
    }
    if (rr <= tol2) {
      status = CONV;
      break;
    }
    if (total >= o.maxit || outer > o.max_outer) {
      status = NOCONV;
      break;
    }
    ++outer;
    k_sh_cg_start<<<gv, kT, 0, s>>>(n, b, q, diag, r, z, p);
    FEM_LAUNCHED();
    FEM_TRY(dots(sh, f->vdim, r, z, nullptr, nullptr, S + 1, comm, s));
    k_sh_copy_scalar<<<1, 1, 0, s>>>(S + 3, S + 1);
    FEM_LAUNCHED();
    status = RUN;
    for (int it = 0; status == RUN; ++it) {
      const int par = it & 1;
      FEM_TRY(apply_raw(sh, f, p, q, true, xz, comm, s));
      FEM_TRY(dots(sh, f->vdim, p, q, nullptr, nullptr, S, comm, s));
      k_sh_cg_update<<<gv, kT, 0, s>>>(n, S, par, x, r, z, p, q, diag);
      FEM_LAUNCHED();
      FEM_TRY(dots(sh, f->vdim, r, z, r, r, S + 1, comm, s));
      FEM_TRY(read_scalars(sh, S, 3, h, s));
      ++total;
      if (!(h[0] > 0.0) || !std::isfinite(h[0]) || !std::isfinite(h[1]) || !std::isfinite(h[2])) {
        status = BREAK;
      } else if (h[2] <= tol2) {
        status = CONV;
      } else if (total >= o.maxit) {
        status = NOCONV;
      } else {
        k_sh_cg_direction<<<gv, kT, 0, s>>>(n, S, par, z, p);
        FEM_LAUNCHED();
      }
    }
    if (status == BREAK) break;
    // confirm with the true residual at the top of the loop
  }
  FEM_CUDA(cudaMemcpyAsync(xio, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  inf.iterations = total;
  inf.outer = outer;
  inf.relres = std::sqrt(rr / bb);
  inf.converged = status == CONV;
  if (info) *info = inf;
  if (status == BREAK) return fem_fail(FEM_EBREAKDOWN, "fem_shard_solve: CG breakdown (p^T A p <= 0 or non-finite)");
  if (status != CONV)
    return fem_fail(FEM_ENOCONV, "fem_shard_solve: no convergence after %d iterations (relres %.3e)", total,
                    inf.relres);
  return FEM_OK;
}
