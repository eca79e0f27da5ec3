// Host side of the C ABI: errors, mesh ingest, the H1 space (global numbering,
// element restriction table and its inverse, boundary DOFs) and form setup.
#include <algorithm>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "fem_internal.h"

static thread_local std::string g_last_error;

fem_status fem_fail(fem_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

extern "C" const char* fem_version(void) { return "fem-gb300 0.1 (sm_103a)"; }
extern "C" const char* fem_last_error(void) { return g_last_error.c_str(); }
extern "C" int fem_supported(int p, int q1d) { return fem_kernels_supported(p, q1d); }

// ----------------------------------------------------------------- mesh ----
static fem_status mesh_create(const double* coords_host, int64_t nv, const int32_t* hex_host, int64_t ne,
                              int dim, fem_mesh** out);

extern "C" fem_status fem_mesh_create(const double* coords_host, int64_t nv,
                                      const int32_t* hex_host, int64_t ne, fem_mesh** out) {
  return mesh_create(coords_host, nv, hex_host, ne, 3, out);
}

extern "C" fem_status fem_mesh2d_create(const double* coords_host, int64_t nv, const int32_t* quad_host,
                                        int64_t ne, fem_mesh** out) {
  return mesh_create(coords_host, nv, quad_host, ne, 2, out);
}

static fem_status mesh_create(const double* coords_host, int64_t nv, const int32_t* hex_host, int64_t ne,
                              int dim, fem_mesh** out) {
  const int nvpe = dim == 3 ? 8 : 4;
  if (!out) return fem_fail(FEM_EINVAL, "fem_mesh_create: out is NULL");
  *out = nullptr;
  if (!coords_host || !hex_host || nv <= 0 || ne <= 0)
    return fem_fail(FEM_EINVAL, "fem_mesh_create: empty mesh or NULL arrays (nv=%lld ne=%lld)",
                    (long long)nv, (long long)ne);
  if (nv >= (int64_t)INT32_MAX || ne >= (int64_t)INT32_MAX / 8)
    return fem_fail(FEM_EUNSUPPORTED, "fem_mesh_create: mesh too large for int32 indices");
  std::vector<uint8_t> used(nv, 0);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t* h = hex_host + nvpe * e;
    for (int a = 0; a < nvpe; ++a) {
      if (h[a] < 0 || h[a] >= nv)
        return fem_fail(FEM_EINVAL, "fem_mesh_create: element %lld vertex %d index %d out of range",
                        (long long)e, a, h[a]);
      for (int b = 0; b < a; ++b)
        if (h[a] == h[b])
          return fem_fail(FEM_EINVAL, "fem_mesh_create: element %lld repeats vertex %d",
                          (long long)e, h[a]);
      used[h[a]] = 1;
    }
  }
  for (int64_t v = 0; v < nv; ++v)
    if (!used[v])
      return fem_fail(FEM_EINVAL, "fem_mesh_create: vertex %lld belongs to no element", (long long)v);
  fem_mesh* m = new fem_mesh();
  m->dim = dim;
  m->nvpe = nvpe;
  m->nv = nv;
  m->ne = ne;
  m->coords.assign(coords_host, coords_host + dim * nv);
  m->hex.assign(hex_host, hex_host + nvpe * ne);
  fem_status st = dev_alloc(&m->d_coords, dim * nv);
  if (st == FEM_OK) st = dev_alloc(&m->d_hex, nvpe * ne);
  if (st == FEM_OK &&
      cudaMemcpy(m->d_coords, coords_host, sizeof(double) * dim * nv, cudaMemcpyHostToDevice) != cudaSuccess)
    st = fem_fail(FEM_ECUDA, "fem_mesh_create: copy of coordinates failed");
  if (st == FEM_OK &&
      cudaMemcpy(m->d_hex, hex_host, sizeof(int32_t) * nvpe * ne, cudaMemcpyHostToDevice) != cudaSuccess)
    st = fem_fail(FEM_ECUDA, "fem_mesh_create: copy of connectivity failed");
  if (st != FEM_OK) {
    fem_mesh_destroy(m);
    return st;
  }
  *out = m;
  return FEM_OK;
}

extern "C" void fem_mesh_destroy(fem_mesh* m) {
  if (!m) return;
  dev_free(m->d_coords);
  dev_free(m->d_hex);
  dev_free(m->d_gnodes);
  delete m;
}

extern "C" fem_status fem_mesh_set_nodes(fem_mesh* m, int k, const double* nodes_host) {
  if (!m) return fem_fail(FEM_EINVAL, "fem_mesh_set_nodes: NULL mesh");
  if (k == 0) {  // back to the vertex (multilinear) geometry
    dev_free(m->d_gnodes);
    m->geo_k = 0;
    return FEM_OK;
  }
  if (k < 1 || k > 8) return fem_fail(FEM_EINVAL, "fem_mesh_set_nodes: order %d not in 1..8", k);
  if (!nodes_host) return fem_fail(FEM_EINVAL, "fem_mesh_set_nodes: NULL nodes");
  // [ne][(k+1)^dim][dim]
  const size_t per = m->dim == 3 ? (size_t)(k + 1) * (k + 1) * (k + 1) * 3 : (size_t)(k + 1) * (k + 1) * 2;
  const size_t n = (size_t)m->ne * per;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(nodes_host[i])) return fem_fail(FEM_EINVAL, "fem_mesh_set_nodes: non-finite coordinate");
  double* d = nullptr;
  FEM_TRY(dev_alloc(&d, n));
  if (cudaMemcpy(d, nodes_host, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
    dev_free(d);
    return fem_fail(FEM_ECUDA, "fem_mesh_set_nodes: copy failed");
  }
  dev_free(m->d_gnodes);
  m->d_gnodes = d;
  m->geo_k = k;
  return FEM_OK;
}

// ---------------------------------------------------------------- space ----
namespace {

// Local entities of the reference hexahedron (vertex indices in VTK order).
const int kEdge[12][2] = {{0, 1}, {1, 2}, {3, 2}, {0, 3}, {4, 5}, {5, 6},
                          {7, 6}, {4, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
// Faces with their 4 corners in cyclic order around the face.
const int kFace[6][4] = {{0, 1, 2, 3}, {0, 1, 5, 4}, {1, 2, 6, 5},
                         {2, 3, 7, 6}, {3, 0, 4, 7}, {4, 5, 6, 7}};
const int kCorner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                           {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

struct Key2 { uint64_t a; uint32_t first; };
struct Key4 { uint64_t a, b; uint32_t first; };

// Ids in order of first appearance: sort (key, appearance), group equal keys,
// then rank the groups by their first appearance.
template <typename K, typename Eq, typename Less>
int64_t first_appearance_ids(std::vector<K>& keys, std::vector<int32_t>& id_of_slot, Eq eq, Less less) {
  const size_t n = keys.size();
  std::vector<uint32_t> order(n);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t x, uint32_t y) { return less(keys[x], keys[y]); });
  std::vector<uint32_t> group_first;   // first appearance (slot) of each group
  std::vector<int32_t> group_of(n);
  for (size_t i = 0; i < n; ++i) {
    if (i == 0 || !eq(keys[order[i]], keys[order[i - 1]])) group_first.push_back(order[i]);
    group_of[order[i]] = (int32_t)group_first.size() - 1;
  }
  const size_t ng = group_first.size();
  std::vector<uint32_t> gorder(ng);
  std::iota(gorder.begin(), gorder.end(), 0u);
  std::sort(gorder.begin(), gorder.end(),
            [&](uint32_t x, uint32_t y) { return group_first[x] < group_first[y]; });
  std::vector<int32_t> rank(ng);
  for (size_t r = 0; r < ng; ++r) rank[gorder[r]] = (int32_t)r;
  id_of_slot.resize(n);
  for (size_t i = 0; i < n; ++i) id_of_slot[i] = rank[group_of[i]];
  return (int64_t)ng;
}

}  // namespace

static fem_status space_finish(fem_space* sp, fem_space** out);
static fem_status space_create_2d(const fem_mesh* mesh, int p, fem_space** out);

// Edge and face ids of a hexahedral mesh (first appearance order), built
// once per mesh and shared by all its spaces: they do not depend on p.
static void mesh_topology(const fem_mesh* mesh) {
  std::lock_guard<std::mutex> lock(mesh->topo_mu);
  if (mesh->topo_done) return;
  const int64_t ne = mesh->ne, nv = mesh->nv;
  const int32_t* hex = mesh->hex.data();
  // edges: key lo*nv+hi, slot e*12+le
  std::vector<Key2> ek((size_t)ne * 12);
  for (int64_t e = 0; e < ne; ++e)
    for (int le = 0; le < 12; ++le) {
      uint64_t a = (uint64_t)hex[8 * e + kEdge[le][0]], b = (uint64_t)hex[8 * e + kEdge[le][1]];
      if (a > b) std::swap(a, b);
      ek[e * 12 + le] = Key2{a * (uint64_t)nv + b, (uint32_t)(e * 12 + le)};
    }
  mesh->n_edges = first_appearance_ids(
      ek, mesh->edge_id, [](const Key2& x, const Key2& y) { return x.a == y.a; },
      [](const Key2& x, const Key2& y) { return x.a < y.a; });
  std::vector<Key2>().swap(ek);
  // faces: key of the sorted 4 corners
  std::vector<Key4> fk((size_t)ne * 6);
  for (int64_t e = 0; e < ne; ++e)
    for (int lf = 0; lf < 6; ++lf) {
      uint64_t v[4];
      for (int c = 0; c < 4; ++c) v[c] = (uint64_t)hex[8 * e + kFace[lf][c]];
      std::sort(v, v + 4);
      fk[e * 6 + lf] = Key4{v[0] * (uint64_t)nv + v[1], v[2] * (uint64_t)nv + v[3], (uint32_t)(e * 6 + lf)};
    }
  mesh->n_faces = first_appearance_ids(
      fk, mesh->face_id, [](const Key4& x, const Key4& y) { return x.a == y.a && x.b == y.b; },
      [](const Key4& x, const Key4& y) { return x.a < y.a || (x.a == y.a && x.b < y.b); });
  mesh->topo_done = true;
}

// Run fn(e0, e1) over [0, ne) in contiguous element ranges on up to 16 host
// threads (each element's work is independent).
template <typename F>
static void for_elements(int64_t ne, F fn) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), 16, ne / 4096 + 1}));
  if (nt == 1) {
    fn((int64_t)0, ne);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t) th.emplace_back(fn, ne * t / nt, ne * (t + 1) / nt);
  for (auto& x : th) x.join();
}

extern "C" fem_status fem_space_create(const fem_mesh* mesh, int p, fem_space** out) {
  if (!out || !mesh) return fem_fail(FEM_EINVAL, "fem_space_create: NULL argument");
  *out = nullptr;
  if (p < 1) return fem_fail(FEM_EINVAL, "fem_space_create: p must be >= 1 (got %d)", p);
  if (p > 8) return fem_fail(FEM_EUNSUPPORTED, "fem_space_create: p = %d > 8 not compiled", p);
  if (mesh->dim == 2) return space_create_2d(mesh, p, out);
  const int64_t ne = mesh->ne, nv = mesh->nv;
  const int D1 = p + 1, nd = D1 * D1 * D1;
  if ((double)ne * nd >= 2147483647.0)
    return fem_fail(FEM_EUNSUPPORTED, "fem_space_create: ne*(p+1)^3 exceeds int32");
  const int32_t* hex = mesh->hex.data();

  mesh_topology(mesh);
  const int64_t n_edges = mesh->n_edges, n_faces = mesh->n_faces;
  const std::vector<int32_t>& edge_id = mesh->edge_id;
  const std::vector<int32_t>& face_id = mesh->face_id;

  const int64_t pm1 = p - 1;
  const int64_t off_e = nv, off_f = off_e + n_edges * pm1, off_i = off_f + n_faces * pm1 * pm1;
  const int64_t ndof = off_i + ne * pm1 * pm1 * pm1;
  if (ndof >= (int64_t)INT32_MAX)
    return fem_fail(FEM_EUNSUPPORTED, "fem_space_create: ndof exceeds int32");

  // Classify the lattice points of the reference element once.
  // type: 0 vertex (ent = corner), 1 edge (ent = local edge), 2 face, 3 interior.
  std::vector<int> ptype(nd), pent(nd);
  for (int k = 0; k < nd; ++k) {
    const int L[3] = {k % D1, (k / D1) % D1, k / (D1 * D1)};
    int onb = 0;
    for (int d = 0; d < 3; ++d) onb += (L[d] == 0 || L[d] == p);
    if (onb == 3) {
      ptype[k] = 0;
      for (int v = 0; v < 8; ++v)
        if (kCorner[v][0] * p == L[0] && kCorner[v][1] * p == L[1] && kCorner[v][2] * p == L[2]) pent[k] = v;
    } else if (onb == 2) {
      ptype[k] = 1;
      for (int le = 0; le < 12; ++le) {
        const int* A = kCorner[kEdge[le][0]];
        const int* B = kCorner[kEdge[le][1]];
        bool on = true;  // on the segment A-B: coordinates where A==B must match
        for (int d = 0; d < 3; ++d)
          if (A[d] == B[d] && A[d] * p != L[d]) on = false;
        if (on) pent[k] = le;
      }
    } else if (onb == 1) {
      ptype[k] = 2;
      for (int lf = 0; lf < 6; ++lf) {
        // the face plane: the coordinate shared by all 4 corners
        for (int d = 0; d < 3; ++d) {
          const int c0 = kCorner[kFace[lf][0]][d];
          bool same = true;
          for (int c = 1; c < 4; ++c) same &= (kCorner[kFace[lf][c]][d] == c0);
          if (same && c0 * p == L[d]) pent[k] = lf;
        }
      }
    } else {
      ptype[k] = 3;
      pent[k] = 0;
    }
  }

  fem_space* sp = new fem_space();
  sp->mesh = mesh;
  sp->p = p;
  sp->D1 = D1;
  sp->nd = nd;
  sp->ne = ne;
  sp->ndof = ndof;
  sp->n_edges = n_edges;
  sp->n_faces = n_faces;
  sp->e2l.assign((size_t)ne * nd, -1);
  for_elements(ne, [&](int64_t e0, int64_t e1) {
  for (int64_t e = e0; e < e1; ++e) {
    const int32_t* h = hex + 8 * e;
    int32_t* row = sp->e2l.data() + (size_t)e * nd;
    for (int k = 0; k < nd; ++k) {
      const int L[3] = {k % D1, (k / D1) % D1, k / (D1 * D1)};
      if (ptype[k] == 0) {
        row[k] = h[pent[k]];
      } else if (ptype[k] == 1) {
        const int le = pent[k];
        int a = kEdge[le][0], b = kEdge[le][1];
        if (h[a] > h[b]) std::swap(a, b);           // a: lower global vertex
        // distance (in lattice steps) from corner a along the edge
        int dist = 0;
        for (int d = 0; d < 3; ++d) dist += std::abs(L[d] - kCorner[a][d] * p);
        row[k] = (int32_t)(off_e + (int64_t)edge_id[e * 12 + le] * pm1 + (dist - 1));
      } else if (ptype[k] == 2) {
        const int lf = pent[k];
        int o = 0;                                  // slot of the lowest global vertex
        for (int c = 1; c < 4; ++c)
          if (h[kFace[lf][c]] < h[kFace[lf][o]]) o = c;
        int na = (o + 1) % 4, nb = (o + 3) % 4;     // cyclic neighbours of o
        if (h[kFace[lf][nb]] < h[kFace[lf][na]]) std::swap(na, nb);
        const int* O = kCorner[kFace[lf][o]];
        const int* A1 = kCorner[kFace[lf][na]];
        const int* A2 = kCorner[kFace[lf][nb]];
        int s = 0, t = 0;                           // projections on the two axes
        for (int d = 0; d < 3; ++d) {
          s += (L[d] - O[d] * p) * (A1[d] - O[d]);
          t += (L[d] - O[d] * p) * (A2[d] - O[d]);
        }
        row[k] = (int32_t)(off_f + (int64_t)face_id[e * 6 + lf] * pm1 * pm1 + (t - 1) * pm1 + (s - 1));
      } else {
        row[k] = (int32_t)(off_i + e * pm1 * pm1 * pm1 + (L[0] - 1) + pm1 * ((L[1] - 1) + pm1 * (L[2] - 1)));
      }
    }
  }
  });

  // boundary DOFs: every lattice point of a face with one adjacent element
  {
    std::vector<int32_t> count(n_faces, 0);
    for (size_t i = 0; i < face_id.size(); ++i) count[face_id[i]]++;
    std::vector<uint8_t> mark(ndof, 0);
    for (int64_t e = 0; e < ne; ++e)
      for (int lf = 0; lf < 6; ++lf) {
        if (count[face_id[e * 6 + lf]] != 1) continue;
        int dplane = -1, val = 0;
        for (int d = 0; d < 3; ++d) {
          const int c0 = kCorner[kFace[lf][0]][d];
          bool same = true;
          for (int c = 1; c < 4; ++c) same &= (kCorner[kFace[lf][c]][d] == c0);
          if (same) { dplane = d; val = c0 * p; }
        }
        for (int k = 0; k < nd; ++k) {
          const int L[3] = {k % D1, (k / D1) % D1, k / (D1 * D1)};
          if (L[dplane] == val) mark[sp->e2l[(size_t)e * nd + k]] = 1;
        }
      }
    for (int64_t i = 0; i < ndof; ++i)
      if (mark[i]) sp->bdr.push_back((int32_t)i);
  }

  return space_finish(sp, out);
}

// Quadrilaterals: vertices, then edges by first appearance (local edges
// (0,1),(1,2),(3,2),(0,3), DOFs from the lower to the higher global
// vertex), then element interiors (lexicographic); boundary DOFs lie on
// edges with one adjacent element.
static fem_status space_create_2d(const fem_mesh* mesh, int p, fem_space** out) {
  static const int kEdge2[4][2] = {{0, 1}, {1, 2}, {3, 2}, {0, 3}};
  static const int kCorner2[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
  const int64_t ne = mesh->ne, nv = mesh->nv;
  const int D1 = p + 1, nd = D1 * D1;
  if ((double)ne * nd >= 2147483647.0)
    return fem_fail(FEM_EUNSUPPORTED, "fem_space_create: ne*(p+1)^2 exceeds int32");
  const int32_t* q4 = mesh->hex.data();
  std::vector<Key2> ek((size_t)ne * 4);
  for (int64_t e = 0; e < ne; ++e)
    for (int le = 0; le < 4; ++le) {
      uint64_t a = (uint64_t)q4[4 * e + kEdge2[le][0]], b = (uint64_t)q4[4 * e + kEdge2[le][1]];
      if (a > b) std::swap(a, b);
      ek[e * 4 + le] = Key2{a * (uint64_t)nv + b, (uint32_t)(e * 4 + le)};
    }
  std::vector<int32_t> edge_id;
  const int64_t n_edges = first_appearance_ids(
      ek, edge_id, [](const Key2& x, const Key2& y) { return x.a == y.a; },
      [](const Key2& x, const Key2& y) { return x.a < y.a; });
  const int64_t pm1 = p - 1;
  const int64_t off_e = nv, off_i = nv + n_edges * pm1, ndof = off_i + ne * pm1 * pm1;
  if (ndof >= (int64_t)INT32_MAX) return fem_fail(FEM_EUNSUPPORTED, "fem_space_create: ndof exceeds int32");
  fem_space* sp = new fem_space();
  sp->mesh = mesh;
  sp->p = p;
  sp->D1 = D1;
  sp->nd = nd;
  sp->ne = ne;
  sp->ndof = ndof;
  sp->n_edges = n_edges;
  sp->e2l.assign((size_t)ne * nd, -1);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t* h = q4 + 4 * e;
    int32_t* row = sp->e2l.data() + (size_t)e * nd;
    for (int k = 0; k < nd; ++k) {
      const int L[2] = {k % D1, k / D1};
      const int onb = (L[0] == 0 || L[0] == p) + (L[1] == 0 || L[1] == p);
      if (onb == 2) {
        for (int v = 0; v < 4; ++v)
          if (kCorner2[v][0] * p == L[0] && kCorner2[v][1] * p == L[1]) row[k] = h[v];
      } else if (onb == 1) {
        for (int le = 0; le < 4; ++le) {
          const int* A = kCorner2[kEdge2[le][0]];
          const int* B = kCorner2[kEdge2[le][1]];
          bool on = true;
          for (int d = 0; d < 2; ++d)
            if (A[d] == B[d] && A[d] * p != L[d]) on = false;
          if (!on) continue;
          int a = kEdge2[le][0], b = kEdge2[le][1];
          if (h[a] > h[b]) std::swap(a, b);
          const int dist = std::abs(L[0] - kCorner2[a][0] * p) + std::abs(L[1] - kCorner2[a][1] * p);
          row[k] = (int32_t)(off_e + (int64_t)edge_id[e * 4 + le] * pm1 + (dist - 1));
        }
      } else {
        row[k] = (int32_t)(off_i + e * pm1 * pm1 + (L[0] - 1) + pm1 * (L[1] - 1));
      }
    }
  }
  std::vector<int32_t> count(n_edges, 0);
  for (size_t i = 0; i < edge_id.size(); ++i) count[edge_id[i]]++;
  std::vector<uint8_t> mark(ndof, 0);
  for (int64_t e = 0; e < ne; ++e)
    for (int le = 0; le < 4; ++le) {
      if (count[edge_id[e * 4 + le]] != 1) continue;
      const int* A = kCorner2[kEdge2[le][0]];
      const int* B = kCorner2[kEdge2[le][1]];
      for (int k = 0; k < nd; ++k) {
        const int L[2] = {k % D1, k / D1};
        bool on = true;
        for (int d = 0; d < 2; ++d)
          if (A[d] == B[d] && A[d] * p != L[d]) on = false;
        if (on) mark[sp->e2l[(size_t)e * nd + k]] = 1;
      }
    }
  for (int64_t i = 0; i < ndof; ++i)
    if (mark[i]) sp->bdr.push_back((int32_t)i);
  return space_finish(sp, out);
}

// Inverse map, GLL nodes and device copies (shared by 2D and 3D).
static fem_status space_finish(fem_space* sp, fem_space** out) {
  const int64_t ndof = sp->ndof, ne = sp->ne;
  const int nd = sp->nd, p = sp->p;
  // inverse map: for each DOF, the E-vector slots e*nd+k holding it, in (e,k) order
  std::vector<int32_t> off(ndof + 1, 0), idx((size_t)ne * nd);
  for (size_t s = 0; s < sp->e2l.size(); ++s) off[sp->e2l[s] + 1]++;
  for (int64_t i = 0; i < ndof; ++i) off[i + 1] += off[i];
  {
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (size_t s = 0; s < sp->e2l.size(); ++s) idx[fill[sp->e2l[s]]++] = (int32_t)s;
  }
  for (int64_t i = 0; i < ndof; ++i)
    if (off[i + 1] == off[i]) {
      fem_space_destroy(sp);
      return fem_fail(FEM_EINVAL, "fem_space_create: DOF %lld has no element", (long long)i);
    }

  fem_gll_nodes(p, sp->nodes);
  fem_status st = dev_alloc(&sp->d_e2l, sp->e2l.size());
  if (st == FEM_OK) st = dev_alloc(&sp->d_l2e_off, off.size());
  if (st == FEM_OK) st = dev_alloc(&sp->d_l2e_idx, idx.size());
  std::vector<int32_t> pos(idx.size());
  for (size_t j = 0; j < idx.size(); ++j) pos[idx[j]] = (int32_t)j;
  if (st == FEM_OK) st = dev_alloc(&sp->d_pos, pos.size());
  if (st == FEM_OK) st = dev_alloc(&sp->d_nodes, sp->nodes.size());
  if (st == FEM_OK) {
    cudaError_t e1 = cudaMemcpy(sp->d_e2l, sp->e2l.data(), sizeof(int32_t) * sp->e2l.size(), cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy(sp->d_l2e_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice);
    cudaError_t e3 = cudaMemcpy(sp->d_l2e_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice);
    if (e3 == cudaSuccess)
      e3 = cudaMemcpy(sp->d_pos, pos.data(), sizeof(int32_t) * pos.size(), cudaMemcpyHostToDevice);
    cudaError_t e4 = cudaMemcpy(sp->d_nodes, sp->nodes.data(), sizeof(double) * sp->nodes.size(), cudaMemcpyHostToDevice);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "fem_space_create: upload of restriction maps failed");
  }
  if (st != FEM_OK) {
    fem_space_destroy(sp);
    return st;
  }
  *out = sp;
  return FEM_OK;
}

extern "C" void fem_space_destroy(fem_space* sp) {
  if (!sp) return;
  dev_free(sp->d_e2l);
  dev_free(sp->d_l2e_off);
  dev_free(sp->d_l2e_idx);
  dev_free(sp->d_pos);
  dev_free(sp->d_nodes);
  dev_free(sp->d_gBn);
  delete sp;
}

extern "C" fem_status fem_space_info(const fem_space* sp, int64_t* ndof, int64_t* nbdr, int64_t* ne,
                                     int* p) {
  if (!sp) return fem_fail(FEM_EINVAL, "fem_space_info: NULL space");
  if (ndof) *ndof = sp->ndof;
  if (nbdr) *nbdr = (int64_t)sp->bdr.size();
  if (ne) *ne = sp->ne;
  if (p) *p = sp->p;
  return FEM_OK;
}

extern "C" fem_status fem_space_boundary_dofs(const fem_space* sp, int32_t* out_host) {
  if (!sp || !out_host) return fem_fail(FEM_EINVAL, "fem_space_boundary_dofs: NULL argument");
  std::memcpy(out_host, sp->bdr.data(), sizeof(int32_t) * sp->bdr.size());
  return FEM_OK;
}

extern "C" fem_status fem_space_element_dofs(const fem_space* sp, int32_t* out_host) {
  if (!sp || !out_host) return fem_fail(FEM_EINVAL, "fem_space_element_dofs: NULL argument");
  std::memcpy(out_host, sp->e2l.data(), sizeof(int32_t) * sp->e2l.size());
  return FEM_OK;
}

extern "C" fem_status fem_space_dof_coords(const fem_space* sp, double* out, void* stream) {
  if (!sp || !out) return fem_fail(FEM_EINVAL, "fem_space_dof_coords: NULL argument");
  return fem_launch_dof_coords(sp, out, (cudaStream_t)stream);
}

// ----------------------------------------------------------------- form ----
static fem_status form_create(const fem_space* sp, int kind, int q1d, const double* coef, const double* beta,
                              const double* mu, void* stream, fem_form** out);

extern "C" fem_status fem_form_create(const fem_space* sp, int kind, int q1d, const double* coef,
                                      void* stream, fem_form** out) {
  if (!sp || !out) return fem_fail(FEM_EINVAL, "fem_form_create: NULL argument");
  *out = nullptr;
  if (kind == FEM_CONVECTION)
    return fem_fail(FEM_EINVAL, "fem_form_create: convection forms need a velocity (fem_form_create_convection)");
  if (kind == FEM_ELASTICITY)
    return fem_fail(FEM_EINVAL, "fem_form_create: elasticity forms need Lame coefficients (fem_form_create_elasticity)");
  if (kind != FEM_MASS && kind != FEM_DIFFUSION)
    return fem_fail(FEM_EINVAL, "fem_form_create: unknown kind %d", kind);
  return form_create(sp, kind, q1d, coef, nullptr, nullptr, stream, out);
}

extern "C" fem_status fem_form_create_convection(const fem_space* sp, int q1d, const double* beta_q,
                                                 const double* coef, void* stream, fem_form** out) {
  if (!sp || !out || !beta_q) return fem_fail(FEM_EINVAL, "fem_form_create_convection: NULL argument");
  *out = nullptr;
  if (sp->mesh->dim != 3) return fem_fail(FEM_EUNSUPPORTED, "fem_form_create_convection: hexahedral meshes only");
  return form_create(sp, FEM_CONVECTION, q1d, coef, beta_q, nullptr, stream, out);
}

extern "C" fem_status fem_form_create_elasticity(const fem_space* sp, int q1d, const double* lambda,
                                                 const double* mu, void* stream, fem_form** out) {
  if (!sp || !out || !lambda || !mu) return fem_fail(FEM_EINVAL, "fem_form_create_elasticity: NULL argument");
  *out = nullptr;
  if (sp->mesh->dim != 3) return fem_fail(FEM_EUNSUPPORTED, "fem_form_create_elasticity: hexahedral meshes only");
  return form_create(sp, FEM_ELASTICITY, q1d, lambda, nullptr, mu, stream, out);
}

static fem_status form_setup(fem_form* f, cudaStream_t s);

// Copy the per-element coefficient (NULL: ones) into the form.
static fem_status copy_coef(fem_form* f, const double* coef, cudaStream_t s) {
  const int64_t ne = f->space->ne;
  if (coef) {
    FEM_CUDA(cudaMemcpyAsync(f->d_coef, coef, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
  } else {
    std::vector<double> ones(ne, 1.0);
    FEM_CUDA(cudaMemcpyAsync(f->d_coef, ones.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaStreamSynchronize(s));
  }
  return FEM_OK;
}

static fem_status form_create(const fem_space* sp, int kind, int q1d, const double* coef, const double* beta,
                              const double* mu, void* stream, fem_form** out) {
  if (!fem_kernels_supported(sp->p, q1d))
    return fem_fail(FEM_EUNSUPPORTED, "fem_form_create: (p=%d, q1d=%d) not compiled", sp->p, q1d);
  FEM_TRY(fem_apply_tables_init());
  if (sp->mesh->dim == 2) FEM_TRY(fem_2d_tables_init());
  if (kind == FEM_ELASTICITY) FEM_TRY(fem_elast_tables_init());
  cudaStream_t s = (cudaStream_t)stream;
  fem_form* f = new fem_form();
  f->space = sp;
  f->kind = kind;
  f->q1d = q1d;
  const int dim = sp->mesh->dim;
  f->nq = dim == 3 ? q1d * q1d * q1d : q1d * q1d;
  f->ncomp = (kind == FEM_DIFFUSION) ? (dim == 3 ? 6 : 3) : kind == FEM_CONVECTION ? 3 : kind == FEM_ELASTICITY ? 12 : 1;
  f->vdim = kind == FEM_ELASTICITY ? 3 : 1;
  std::vector<double> pts, wts, B, G;
  fem_gauss_rule(q1d, pts, wts);
  fem_lagrange_tables(sp->nodes, pts, B, G);
  std::vector<float> B32(B.begin(), B.end()), G32(G.begin(), G.end());
  // double-float pairs: hi = fl32(v), lo = fl32(v - hi)
  std::vector<float> Bdf(2 * B.size()), Gdf(2 * G.size());
  for (size_t i = 0; i < B.size(); ++i) {
    Bdf[2 * i] = (float)B[i];
    Bdf[2 * i + 1] = (float)(B[i] - (double)Bdf[2 * i]);
    Gdf[2 * i] = (float)G[i];
    Gdf[2 * i + 1] = (float)(G[i] - (double)Gdf[2 * i]);
  }
  fem_status st = FEM_OK;
  auto up = [&](auto** dst, const auto& src) {
    if (st != FEM_OK) return;
    st = dev_alloc(dst, src.size());
    if (st == FEM_OK &&
        cudaMemcpy(*dst, src.data(), sizeof(src[0]) * src.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "fem_form_create: table upload failed");
  };
  up(&f->d_B, B);
  up(&f->d_G, G);
  up(&f->d_B32, B32);
  up(&f->d_G32, G32);
  up(&f->d_Bdf, Bdf);
  up(&f->d_Gdf, Gdf);
  up(&f->d_qpts, pts);
  up(&f->d_qwts, wts);
  if (st == FEM_OK) st = dev_alloc(&f->d_coef, (size_t)sp->ne);
  if (st == FEM_OK) st = dev_alloc(&f->d_D, (size_t)sp->ne * f->ncomp * f->nq + 2);  // +16 bytes slack
  if (st == FEM_OK) st = dev_alloc((double**)&f->d_ye, (size_t)f->vdim * sp->ne * sp->nd);
  if (st == FEM_OK && mu) {
    st = dev_alloc(&f->d_mu, (size_t)sp->ne);
    if (st == FEM_OK &&
        cudaMemcpyAsync(f->d_mu, mu, sizeof(double) * sp->ne, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "fem_form_create: mu copy failed");
  }
  if (st == FEM_OK) st = dev_alloc(&f->d_flag, 4);
  if (st == FEM_OK && cudaMallocHost((void**)&f->h_pinned, 64) != cudaSuccess)
    st = fem_fail(FEM_ENOMEM, "fem_form_create: pinned host allocation failed");
  if (st == FEM_OK && beta) {
    const size_t nb = (size_t)sp->ne * f->nq * 3;
    st = dev_alloc(&f->d_beta, nb);
    if (st == FEM_OK && cudaMemcpyAsync(f->d_beta, beta, sizeof(double) * nb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      st = fem_fail(FEM_ECUDA, "fem_form_create: velocity copy failed");
  }
  if (st != FEM_OK) {
    fem_form_destroy(f);
    return st;
  }
  st = copy_coef(f, coef, s);
  if (st == FEM_OK) st = form_setup(f, s);
  if (st != FEM_OK) {
    fem_form_destroy(f);
    return st;
  }
  *out = f;
  return FEM_OK;
}

fem_status fem_form_geo_tables(const fem_form* fc) {
  fem_form* f = const_cast<fem_form*>(fc);
  const fem_mesh* m = f->space->mesh;
  if (m->geo_k <= 0 || f->geo_k == m->geo_k) return FEM_OK;
  std::vector<double> nk, pts, wts, B, G;
  fem_gll_nodes(m->geo_k, nk);
  fem_gauss_rule(f->q1d, pts, wts);
  fem_lagrange_tables(nk, pts, B, G);  // [q1d][k+1]
  dev_free(f->d_gB);
  dev_free(f->d_gG);
  FEM_TRY(dev_alloc(&f->d_gB, B.size()));
  FEM_TRY(dev_alloc(&f->d_gG, G.size()));
  FEM_CUDA(cudaMemcpy(f->d_gB, B.data(), sizeof(double) * B.size(), cudaMemcpyHostToDevice));
  FEM_CUDA(cudaMemcpy(f->d_gG, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice));
  f->geo_k = m->geo_k;
  return FEM_OK;
}

extern "C" fem_status fem_form_set_coef(fem_form* f, const double* coef, void* stream) {
  if (!f) return fem_fail(FEM_EINVAL, "fem_form_set_coef: NULL form");
  if (f->kind == FEM_ELASTICITY) return fem_fail(FEM_EINVAL, "fem_form_set_coef: elasticity forms take fem_form_set_lame");
  cudaStream_t s = (cudaStream_t)stream;
  FEM_TRY(copy_coef(f, coef, s));
  return form_setup(f, s);
}

extern "C" fem_status fem_form_set_lame(fem_form* f, const double* lambda, const double* mu, void* stream) {
  if (!f || !lambda || !mu) return fem_fail(FEM_EINVAL, "fem_form_set_lame: NULL argument");
  if (f->kind != FEM_ELASTICITY) return fem_fail(FEM_EINVAL, "fem_form_set_lame: not an elasticity form");
  cudaStream_t s = (cudaStream_t)stream;
  FEM_TRY(copy_coef(f, lambda, s));
  FEM_CUDA(cudaMemcpyAsync(f->d_mu, mu, sizeof(double) * f->space->ne, cudaMemcpyDeviceToDevice, s));
  return form_setup(f, s);
}

static fem_status form_setup(fem_form* f, cudaStream_t s) {
  FEM_CUDA(cudaMemsetAsync(f->d_flag, 0, sizeof(int) * 4, s));
  FEM_TRY(fem_launch_setup(f, s));
  FEM_CUDA(cudaMemcpyAsync(f->h_pinned, f->d_flag, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  dev_free(f->d_D32);  // any float / double-float copy is stale now
  dev_free(f->d_Ddf);
  if (f->h_pinned[0] != 0)
    return fem_fail(FEM_EINVERTED, "fem_form: det J <= 0 at a quadrature point of element %d",
                    f->h_pinned[1]);
  return FEM_OK;
}

extern "C" fem_status fem_form_set_velocity(fem_form* f, const double* beta, void* stream) {
  if (!f || !beta) return fem_fail(FEM_EINVAL, "fem_form_set_velocity: NULL argument");
  if (f->kind != FEM_CONVECTION) return fem_fail(FEM_EINVAL, "fem_form_set_velocity: not a convection form");
  cudaStream_t s = (cudaStream_t)stream;
  FEM_CUDA(cudaMemcpyAsync(f->d_beta, beta, sizeof(double) * (size_t)f->space->ne * f->nq * 3,
                           cudaMemcpyDeviceToDevice, s));
  return form_setup(f, s);
}

extern "C" void fem_form_destroy(fem_form* f) {
  if (!f) return;
  dev_free(f->d_coef);
  dev_free(f->d_mu);
  dev_free(f->d_D);
  dev_free(f->d_D32);
  dev_free(f->d_B);
  dev_free(f->d_G);
  dev_free(f->d_B32);
  dev_free(f->d_G32);
  dev_free(f->d_Bdf);
  dev_free(f->d_Gdf);
  dev_free(f->d_Ddf);
  dev_free(f->d_gB);
  dev_free(f->d_gG);
  dev_free(f->d_beta);
  dev_free(f->d_qpts);
  dev_free(f->d_qwts);
  if (f->d_ye) cudaFree(f->d_ye);
  dev_free(f->d_ess_mask);
  dev_free(f->d_ess);
  dev_free(f->d_flag);
  dev_free(f->d_work64);
  dev_free(f->d_work32);
  dev_free(f->d_red);
  if (f->h_pinned) cudaFreeHost(f->h_pinned);
  delete f;
}

extern "C" fem_status fem_form_set_essential(fem_form* f, const int32_t* ess, int64_t n, void* stream) {
  if (!f) return fem_fail(FEM_EINVAL, "fem_form_set_essential: NULL form");
  if (n < 0 || (n > 0 && !ess)) return fem_fail(FEM_EINVAL, "fem_form_set_essential: bad list");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ndof = fem_form_len(f);
  if (!f->d_ess_mask) FEM_TRY(dev_alloc(&f->d_ess_mask, (size_t)ndof));
  dev_free(f->d_ess);
  f->n_ess = n;
  FEM_CUDA(cudaMemsetAsync(f->d_ess_mask, 0, (size_t)ndof, s));
  if (n > 0) {
    FEM_TRY(dev_alloc(&f->d_ess, (size_t)n));
    FEM_CUDA(cudaMemcpyAsync(f->d_ess, ess, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    // mark the mask on the device; out-of-range ids are reported through the flag
    FEM_CUDA(cudaMemsetAsync(f->d_flag, 0, sizeof(int) * 4, s));
    FEM_TRY(fem_launch_mark_ess(f, s));
    FEM_CUDA(cudaMemcpyAsync(f->h_pinned, f->d_flag, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    FEM_CUDA(cudaStreamSynchronize(s));
    if (f->h_pinned[2] != 0)
      return fem_fail(FEM_EINVAL, "fem_form_set_essential: DOF id out of range");
  }
  return FEM_OK;
}

// ------------------------------------------------------ multigrid (host) ----
// Entity signature of local node k of a (D1)^3 lattice: per axis 0 (at 0),
// 2 (at D1-1), 1 (inside); s = s_x + 3 s_y + 9 s_z.
static int lattice_signature(int k, int D1) {
  const int L[3] = {k % D1, (k / D1) % D1, k / (D1 * D1)};
  int s = 0, w = 1;
  for (int d = 0; d < 3; ++d, w *= 3) s += w * (L[d] == 0 ? 0 : L[d] == D1 - 1 ? 2 : 1);
  return s;
}

// Coarse essential DOFs of the p-multigrid hierarchy (k_mg.cu): a coarse
// DOF is essential iff every fine DOF of the same mesh entity (vertex, edge,
// face or interior of one element) is. essf: the fine mask of one component
// ([sf->ndof]); returns the coarse DOF ids, ascending.
std::vector<int32_t> fem_coarse_essential(const fem_space* sf, const uint8_t* essf, const fem_space* sc) {
  const int Df = sf->D1, Dc = sc->D1, ndf = sf->nd, ndc = sc->nd;
  std::vector<int> sigf(ndf), sigc(ndc);
  for (int k = 0; k < ndf; ++k) sigf[k] = lattice_signature(k, Df);
  for (int k = 0; k < ndc; ++k) sigc[k] = lattice_signature(k, Dc);
  std::vector<uint8_t> mark(sc->ndof, 0);
  for (int64_t e = 0; e < sf->ne; ++e) {
    int all[27];
    for (int s = 0; s < 27; ++s) all[s] = 1;
    const int32_t* rf = sf->e2l.data() + (size_t)e * ndf;
    for (int k = 0; k < ndf; ++k)
      if (!essf[rf[k]]) all[sigf[k]] = 0;
    const int32_t* rc = sc->e2l.data() + (size_t)e * ndc;
    for (int k = 0; k < ndc; ++k)
      if (all[sigc[k]]) mark[rc[k]] = 1;
  }
  std::vector<int32_t> out;
  for (int64_t i = 0; i < sc->ndof; ++i)
    if (mark[i]) out.push_back((int32_t)i);
  return out;
}

