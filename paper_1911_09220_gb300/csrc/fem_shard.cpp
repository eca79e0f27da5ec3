// Host side of the sharded operator: the element partition and the plan of
// one rank's shard (local mesh and space, local -> global DOF map,
// ownership, neighbours, exchange slots and the combine table).
//
// The paper's parallel operator is A = P^T G^T B^T D B G P (Sec. 4.3): each
// rank runs the element operator on its own elements; P^T sums the partial
// results of DOFs that several ranks hold into one value and P hands that
// value back to every holder (the parallel assembly of FormLinearSystem,
// Sec. 5.1). The plan below fixes, for every DOF a rank shares, which
// neighbours hold it, where its partials travel, and the order (ascending
// rank) in which they are added, so every holder computes the same sum.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "fem_internal.h"

namespace {

int lowest_bit(uint64_t m) {
  int b = 0;
  while (!(m & 1u)) {
    m >>= 1;
    ++b;
  }
  return b;
}

}  // namespace

extern "C" fem_status fem_partition_slabs(const fem_mesh* m, int nparts, int32_t* part_host) {
  if (!m || !part_host) return fem_fail(FEM_EINVAL, "fem_partition_slabs: NULL argument");
  const int64_t ne = m->ne;
  if (nparts < 1 || nparts > ne)
    return fem_fail(FEM_EINVAL, "fem_partition_slabs: nparts = %d for %lld elements", nparts, (long long)ne);
  const int dim = m->dim, nvpe = m->nvpe;
  std::vector<double> cen((size_t)ne * dim, 0.0);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t e = 0; e < ne; ++e) {
    for (int a = 0; a < nvpe; ++a) {
      const int32_t v = m->hex[(size_t)e * nvpe + a];
      for (int d = 0; d < dim; ++d) cen[(size_t)e * dim + d] += m->coords[(size_t)v * dim + d];
    }
    for (int d = 0; d < dim; ++d) {
      const double c = cen[(size_t)e * dim + d] / nvpe;
      cen[(size_t)e * dim + d] = c;
      lo[d] = std::min(lo[d], c);
      hi[d] = std::max(hi[d], c);
    }
  }
  int axis = 0;
  for (int d = 1; d < dim; ++d)
    if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
  std::vector<int64_t> order(ne);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const double ca = cen[(size_t)a * dim + axis], cb = cen[(size_t)b * dim + axis];
    return ca < cb || (ca == cb && a < b);
  });
  const int64_t base = ne / nparts, extra = ne % nparts;
  int64_t pos = 0;
  for (int r = 0; r < nparts; ++r) {
    const int64_t len = base + (r < extra ? 1 : 0);
    for (int64_t i = 0; i < len; ++i) part_host[order[pos++]] = r;
  }
  return FEM_OK;
}

static fem_status upload_plan(fem_shard* sh);

extern "C" fem_status fem_shard_create(const fem_space* gs, const int32_t* part, int nparts, int rank,
                                       fem_shard** out) {
  if (!out) return fem_fail(FEM_EINVAL, "fem_shard_create: out is NULL");
  *out = nullptr;
  if (!gs || !part) return fem_fail(FEM_EINVAL, "fem_shard_create: NULL argument");
  if (nparts < 1 || nparts > 64 || rank < 0 || rank >= nparts)
    return fem_fail(FEM_EINVAL, "fem_shard_create: rank %d of %d parts (1 <= nparts <= 64)", rank, nparts);
  const fem_mesh* gm = gs->mesh;
  if (gm->geo_k > 0) return fem_fail(FEM_EUNSUPPORTED, "fem_shard_create: curved (nodal) meshes are not sharded");
  const int64_t ne = gs->ne;
  const int nd = gs->nd, nvpe = gm->nvpe, dim = gm->dim;
  for (int64_t e = 0; e < ne; ++e)
    if (part[e] < 0 || part[e] >= nparts)
      return fem_fail(FEM_EINVAL, "fem_shard_create: element %lld in part %d", (long long)e, part[e]);

  fem_shard* sh = new fem_shard();
  sh->nparts = nparts;
  sh->rank = rank;
  sh->ndof_global = gs->ndof;
  for (int64_t e = 0; e < ne; ++e)
    if (part[e] == rank) sh->elems.push_back(e);
  if (sh->elems.empty()) {
    delete sh;
    return fem_fail(FEM_EINVAL, "fem_shard_create: rank %d has no elements", rank);
  }
  // local mesh: the shard's vertices in ascending global number
  const int64_t nel = (int64_t)sh->elems.size();
  std::vector<int32_t> vmap(gm->nv, -1);
  for (int64_t e : sh->elems)
    for (int a = 0; a < nvpe; ++a) vmap[gm->hex[(size_t)e * nvpe + a]] = 0;
  std::vector<double> lc;
  int32_t nlv = 0;
  for (int64_t v = 0; v < gm->nv; ++v)
    if (vmap[v] == 0) {
      vmap[v] = nlv++;
      for (int d = 0; d < dim; ++d) lc.push_back(gm->coords[(size_t)v * dim + d]);
    }
  std::vector<int32_t> lh((size_t)nel * nvpe);
  for (int64_t j = 0; j < nel; ++j)
    for (int a = 0; a < nvpe; ++a) lh[(size_t)j * nvpe + a] = vmap[gm->hex[(size_t)sh->elems[j] * nvpe + a]];
  fem_status st = dim == 3 ? fem_mesh_create(lc.data(), nlv, lh.data(), nel, &sh->lmesh)
                           : fem_mesh2d_create(lc.data(), nlv, lh.data(), nel, &sh->lmesh);
  if (st == FEM_OK) st = fem_space_create(sh->lmesh, gs->p, &sh->lspace);
  if (st != FEM_OK) {
    fem_shard_destroy(sh);
    return st;
  }
  const fem_space* ls = sh->lspace;
  const int64_t nl = ls->ndof;
  // local -> global DOF: the same (element, local node) slot in both spaces
  // (an element keeps its vertex order, so its local frame is the same)
  sh->l2g.assign(nl, -1);
  for (int64_t j = 0; j < nel; ++j) {
    const int64_t e = sh->elems[j];
    for (int k = 0; k < nd; ++k) {
      const int32_t li = ls->e2l[(size_t)j * nd + k];
      const int64_t g = gs->e2l[(size_t)e * nd + k];
      if (sh->l2g[li] >= 0 && sh->l2g[li] != g) {
        fem_shard_destroy(sh);
        return fem_fail(FEM_EINVAL, "fem_shard_create: local DOF %d maps to global %lld and %lld", li,
                        (long long)sh->l2g[li], (long long)g);
      }
      sh->l2g[li] = g;
    }
  }
  // the ranks holding each global DOF
  std::vector<uint64_t> holders(gs->ndof, 0);
  for (int64_t e = 0; e < ne; ++e) {
    const uint64_t bit = (uint64_t)1 << part[e];
    for (int k = 0; k < nd; ++k) holders[gs->e2l[(size_t)e * nd + k]] |= bit;
  }
  sh->owned.assign(nl, 0);
  uint64_t others = 0;
  const uint64_t me = (uint64_t)1 << rank;
  for (int64_t i = 0; i < nl; ++i) {
    const uint64_t h = holders[sh->l2g[i]];
    if (lowest_bit(h) == rank) {
      sh->owned[i] = 1;
      sh->n_owned++;
    }
    others |= h & ~me;
  }
  for (int r = 0; r < nparts; ++r)
    if (others & ((uint64_t)1 << r)) sh->nbr.push_back(r);
  const int nn = (int)sh->nbr.size();
  // slots: per neighbour, the local DOFs it also holds, ascending global DOF
  std::vector<int64_t> by_global(nl);
  std::iota(by_global.begin(), by_global.end(), 0);
  std::sort(by_global.begin(), by_global.end(), [&](int64_t a, int64_t b) { return sh->l2g[a] < sh->l2g[b]; });
  sh->slot_off.assign(nn + 1, 0);
  std::vector<std::vector<int32_t>> slot_of(nn);  // slot of each local DOF, per neighbour (-1: none)
  for (int k = 0; k < nn; ++k) {
    const uint64_t bit = (uint64_t)1 << sh->nbr[k];
    slot_of[k].assign(nl, -1);
    for (int64_t t = 0; t < nl; ++t) {
      const int64_t i = by_global[t];
      if (holders[sh->l2g[i]] & bit) {
        slot_of[k][i] = (int32_t)sh->slot_dof.size();
        sh->slot_dof.push_back((int32_t)i);
      }
    }
    sh->slot_off[k + 1] = (int64_t)sh->slot_dof.size();
  }
  // combine table: DOFs held by more than one rank, partials in rank order
  std::vector<int> nbr_index(nparts, -1);
  for (int k = 0; k < nn; ++k) nbr_index[sh->nbr[k]] = k;
  sh->comb_off.push_back(0);
  for (int64_t i = 0; i < nl; ++i) {
    const uint64_t h = holders[sh->l2g[i]];
    if (!(h & ~me)) continue;
    sh->comb_dof.push_back((int32_t)i);
    for (int r = 0; r < nparts; ++r) {
      if (!(h & ((uint64_t)1 << r))) continue;
      sh->comb_src.push_back(r == rank ? -1 : slot_of[nbr_index[r]][i]);
    }
    sh->comb_off.push_back((int32_t)sh->comb_src.size());
  }
  // exchange buffer offsets (doubles) for scalar and 3-component vectors
  sh->xoff1.assign(nn + 1, 0);
  sh->xoff3.assign(nn + 1, 0);
  for (int k = 0; k <= nn; ++k) {
    sh->xoff1[k] = sh->slot_off[k];
    sh->xoff3[k] = 3 * sh->slot_off[k];
  }
  st = upload_plan(sh);
  if (st != FEM_OK) {
    fem_shard_destroy(sh);
    return st;
  }
  *out = sh;
  return FEM_OK;
}

template <typename T>
static fem_status upload(T** d, const std::vector<T>& h) {
  if (h.empty()) return FEM_OK;
  FEM_TRY(dev_alloc(d, h.size()));
  if (cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return fem_fail(FEM_ECUDA, "fem_shard_create: upload failed");
  return FEM_OK;
}

static fem_status upload_plan(fem_shard* sh) {
  const int64_t nslots = (int64_t)sh->slot_dof.size();
  std::vector<int32_t> slot_nbr(nslots);
  for (size_t k = 0; k + 1 < sh->slot_off.size(); ++k)
    for (int64_t t = sh->slot_off[k]; t < sh->slot_off[k + 1]; ++t) slot_nbr[t] = (int32_t)k;
  FEM_TRY(upload(&sh->d_l2g, sh->l2g));
  FEM_TRY(upload(&sh->d_owned, sh->owned));
  FEM_TRY(upload(&sh->d_slot_dof, sh->slot_dof));
  FEM_TRY(upload(&sh->d_slot_nbr, slot_nbr));
  FEM_TRY(upload(&sh->d_slot_off, sh->slot_off));
  FEM_TRY(upload(&sh->d_comb_dof, sh->comb_dof));
  FEM_TRY(upload(&sh->d_comb_off, sh->comb_off));
  FEM_TRY(upload(&sh->d_comb_src, sh->comb_src));
  if (nslots > 0) {
    FEM_TRY(dev_alloc(&sh->d_send, (size_t)3 * nslots));
    FEM_TRY(dev_alloc(&sh->d_recv, (size_t)3 * nslots));
  }
  return FEM_OK;
}

extern "C" void fem_shard_destroy(fem_shard* sh) {
  if (!sh) return;
  dev_free(sh->d_l2g);
  dev_free(sh->d_owned);
  dev_free(sh->d_slot_dof);
  dev_free(sh->d_slot_nbr);
  dev_free(sh->d_slot_off);
  dev_free(sh->d_comb_dof);
  dev_free(sh->d_comb_off);
  dev_free(sh->d_comb_src);
  dev_free(sh->d_send);
  dev_free(sh->d_recv);
  dev_free(sh->d_work);
  dev_free(sh->d_red);
  if (sh->h_pinned) cudaFreeHost(sh->h_pinned);
  if (sh->lspace) fem_space_destroy(sh->lspace);
  if (sh->lmesh) fem_mesh_destroy(sh->lmesh);
  delete sh;
}

extern "C" const fem_space* fem_shard_space(const fem_shard* sh) { return sh ? sh->lspace : nullptr; }

extern "C" fem_status fem_shard_info(const fem_shard* sh, int64_t* ne_local, int64_t* ndof_local,
                                     int64_t* ndof_owned, int* nnbr, int64_t* nslots, int64_t* ndof_global) {
  if (!sh) return fem_fail(FEM_EINVAL, "fem_shard_info: NULL shard");
  if (ne_local) *ne_local = (int64_t)sh->elems.size();
  if (ndof_local) *ndof_local = sh->lspace->ndof;
  if (ndof_owned) *ndof_owned = sh->n_owned;
  if (nnbr) *nnbr = (int)sh->nbr.size();
  if (nslots) *nslots = (int64_t)sh->slot_dof.size();
  if (ndof_global) *ndof_global = sh->ndof_global;
  return FEM_OK;
}

template <typename T>
static void copy_out(T* dst, const std::vector<T>& v) {
  if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(T) * v.size());
}

extern "C" fem_status fem_shard_tables(const fem_shard* sh, int64_t* elems, int64_t* l2g, uint8_t* owned,
                                       int32_t* nbr, int64_t* slot_off, int32_t* slot_dof) {
  if (!sh) return fem_fail(FEM_EINVAL, "fem_shard_tables: NULL shard");
  copy_out(elems, sh->elems);
  copy_out(l2g, sh->l2g);
  copy_out(owned, sh->owned);
  copy_out(nbr, sh->nbr);
  copy_out(slot_off, sh->slot_off);
  copy_out(slot_dof, sh->slot_dof);
  return FEM_OK;
}

extern "C" fem_status fem_shard_combine_table(const fem_shard* sh, int64_t* nshared, int64_t* nentries,
                                              int32_t* comb_dof, int32_t* comb_off, int32_t* comb_src) {
  if (!sh) return fem_fail(FEM_EINVAL, "fem_shard_combine_table: NULL shard");
  if (nshared) *nshared = (int64_t)sh->comb_dof.size();
  if (nentries) *nentries = (int64_t)sh->comb_src.size();
  copy_out(comb_dof, sh->comb_dof);
  copy_out(comb_off, sh->comb_off);
  copy_out(comb_src, sh->comb_src);
  return FEM_OK;
}

extern "C" fem_status fem_shard_localize(const fem_shard* sh, const int32_t* global_host, int64_t n,
                                         int32_t* out_host) {
  if (!sh || (n > 0 && (!global_host || !out_host))) return fem_fail(FEM_EINVAL, "fem_shard_localize: NULL argument");
  std::vector<int64_t> order(sh->l2g.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return sh->l2g[a] < sh->l2g[b]; });
  for (int64_t i = 0; i < n; ++i) {
    const int64_t g = global_host[i];
    auto it = std::lower_bound(order.begin(), order.end(), g,
                               [&](int64_t a, int64_t val) { return sh->l2g[a] < val; });
    out_host[i] = (it != order.end() && sh->l2g[*it] == g) ? (int32_t)*it : -1;
  }
  return FEM_OK;
}
