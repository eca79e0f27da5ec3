"""Global H1 DOF numbering, element DOF lists and boundary DOFs (oracle; test
infrastructure only).

Sec. 3.4 ("Finite Element Spaces") fixes the order of global enumeration:
all vertex DOFs, then all edge DOFs edge by edge along a fixed direction,
then all face DOFs face by face in a fixed orientation, then element
interiors element by element. It does not say which direction or
orientation; the reading used here (and by the CUDA library) is:

* vertex DOF id = vertex index;
* edges and faces are numbered in order of first appearance when scanning
  elements in order and, inside an element, its 12 edges / 6 faces in the
  local order EDGES / FACES below;
* an edge's p-1 interior DOFs run from its lower to its higher global vertex;
* a face's (p-1)^2 interior DOFs are listed row by row in the frame whose
  origin is the face's lowest global vertex O, whose first axis points to the
  lower-numbered of O's two face neighbours and whose second axis points to
  the other (first axis fastest);
* element interiors in element order, lexicographic (x fastest).

Inside an element the local DOFs are lexicographic on the (p+1)^3 lattice,
first reference coordinate fastest.

This implementation identifies each lattice point of each element by the
integer trilinear weights of the 8 corners at that point: the set of corners
with non-zero weight names the entity (1 corner: vertex, 2: edge, 4: face,
8: interior) and the weights give the position inside it, so two elements
that share an entity agree on a point whatever their local orientation.
"""

import numpy as np

CORNERS = np.array(
    [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
     [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)

EDGES = np.array([[0, 1], [1, 2], [3, 2], [0, 3],
                  [4, 5], [5, 6], [7, 6], [4, 7],
                  [0, 4], [1, 5], [2, 6], [3, 7]], dtype=np.int64)

FACES = np.array([[0, 1, 2, 3], [0, 1, 5, 4], [1, 2, 6, 5],
                  [2, 3, 7, 6], [3, 0, 4, 7], [4, 5, 6, 7]], dtype=np.int64)


def lattice(p):
    """Reference lattice indices [(p+1)^3, 3], first coordinate fastest."""
    r = np.arange(p + 1)
    i3, i2, i1 = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([i1.ravel(), i2.ravel(), i3.ravel()], axis=1)


def corner_weights(p):
    """W[point, v] = prod_d (i_d if corner v has c_d = 1 else p - i_d), the
    trilinear weight of corner v at the lattice point, times p^3."""
    L = lattice(p)
    W = np.ones((L.shape[0], 8), dtype=np.int64)
    for v in range(8):
        for d in range(3):
            W[:, v] *= np.where(CORNERS[v, d] == 1, L[:, d], p - L[:, d])
    return W


def _first_appearance_ids(keys):
    """Give each distinct row of `keys` an id in order of its first row."""
    _, first, inverse = np.unique(keys, axis=0, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    return rank[inverse.ravel()], order.size


def build(hexes, p, nv=None):
    """Return dict with e2l [E, (p+1)^3] int64, ndof, counts and entity ids."""
    hexes = np.asarray(hexes, dtype=np.int64)
    E = hexes.shape[0]
    if nv is None:
        nv = int(hexes.max()) + 1
    D = p + 1
    W = corner_weights(p)
    nnz = (W > 0).sum(axis=1)

    # edges: keys (lo, hi) of global vertex ids, E*12 rows in scan order
    ge = hexes[:, EDGES]                                   # [E,12,2]
    ekeys = np.sort(ge, axis=2).reshape(-1, 2)
    edge_id, n_edges = _first_appearance_ids(ekeys)
    edge_id = edge_id.reshape(E, 12)

    gf = hexes[:, FACES]                                   # [E,6,4]
    fkeys = np.sort(gf, axis=2).reshape(-1, 4)
    face_id, n_faces = _first_appearance_ids(fkeys)
    face_id = face_id.reshape(E, 6)

    pm1 = p - 1
    off_e = nv
    off_f = off_e + n_edges * pm1
    off_i = off_f + n_faces * pm1 * pm1
    ndof = off_i + E * pm1 ** 3

    e2l = np.full((E, D ** 3), -1, dtype=np.int64)
    L = lattice(p)
    for k in range(D ** 3):
        nzv = np.nonzero(W[k])[0]
        if nnz[k] == 1:
            e2l[:, k] = hexes[:, nzv[0]]
        elif nnz[k] == 2:
            a, b = nzv
            le = [i for i in range(12) if set(EDGES[i]) == {a, b}][0]
            ga, gb = hexes[:, a], hexes[:, b]
            # position counted from the lower global vertex, in units of 1/p
            pos = np.where(ga < gb, W[k, b], W[k, a]) // (p * p)
            e2l[:, k] = off_e + edge_id[:, le] * pm1 + (pos - 1)
        elif nnz[k] == 4:
            lf = [i for i in range(6) if set(FACES[i]) == set(nzv)][0]
            corners = FACES[lf]
            g = hexes[:, corners]                         # [E,4]
            o = np.argmin(g, axis=1)                      # local slot of origin
            s_list = np.zeros(E, dtype=np.int64)
            t_list = np.zeros(E, dtype=np.int64)
            # neighbours of the origin: corners differing in one coordinate
            cc = CORNERS[corners]                         # [4,3]
            adj = (np.abs(cc[:, None, :] - cc[None, :, :]).sum(axis=2) == 1)   # [4,4]
            for slot in range(4):
                sel = o == slot
                if not np.any(sel):
                    continue
                nb = np.nonzero(adj[slot])[0]             # two neighbour slots
                diag = [s for s in range(4) if s != slot and s not in nb][0]
                g_nb = g[sel][:, nb]                      # [m,2]
                first_is_0 = g_nb[:, 0] < g_nb[:, 1]
                n1 = np.where(first_is_0, nb[0], nb[1])
                n2 = np.where(first_is_0, nb[1], nb[0])
                wk = W[k, corners]                        # weights of the 4 corners
                s_list[sel] = (wk[n1] + wk[diag]) // (p * p)
                t_list[sel] = (wk[n2] + wk[diag]) // (p * p)
            e2l[:, k] = off_f + face_id[:, lf] * pm1 * pm1 + (t_list - 1) * pm1 + (s_list - 1)
        else:
            i1, i2, i3 = L[k]
            e2l[:, k] = off_i + np.arange(E) * pm1 ** 3 + (i1 - 1) + pm1 * ((i2 - 1) + pm1 * (i3 - 1))
    assert (e2l >= 0).all()

    # boundary faces: faces with exactly one adjacent element
    counts = np.bincount(face_id.ravel(), minlength=n_faces)
    bnd_face = counts[face_id] == 1                        # [E,6]
    bmask = np.zeros(ndof, dtype=bool)
    for lf in range(6):
        pts = [k for k in range(D ** 3) if set(np.nonzero(W[k])[0]) <= set(FACES[lf])]
        rows = np.nonzero(bnd_face[:, lf])[0]
        if rows.size:
            bmask[e2l[np.ix_(rows, pts)].ravel()] = True
    return {
        "e2l": e2l, "ndof": ndof, "nv": nv, "n_edges": n_edges, "n_faces": n_faces,
        "boundary_mask": bmask, "boundary_dofs": np.nonzero(bmask)[0],
    }


def dof_coords(coords, hexes, p, e2l, nodes):
    """Physical location of every global DOF: the trilinear map of its element
    evaluated at the GLL node of its lattice point (Sec. 3.1, mesh map
    x(xhat) = sum_i x_i w_i(xhat) with trilinear w_i)."""
    coords = np.asarray(coords, dtype=np.float64)
    hexes = np.asarray(hexes, dtype=np.int64)
    L = lattice(p)
    xi = nodes[L]                                         # [D^3, 3]
    N = np.ones((L.shape[0], 8))
    for v in range(8):
        for d in range(3):
            N[:, v] *= np.where(CORNERS[v, d] == 1, xi[:, d], 1.0 - xi[:, d])
    X = coords[hexes]                                     # [E,8,3]
    pts = np.einsum("kv,evr->ekr", N, X)                  # [E,D^3,3]
    ndof = int(e2l.max()) + 1
    out = np.zeros((ndof, 3))
    out[e2l.ravel()] = pts.reshape(-1, 3)
    return out
