"""Structured-topology hexahedral meshes handed on as unstructured arrays.

Local vertex order of a hexahedron (the VTK / MFEM convention): bottom face
0-1-2-3 counter-clockwise seen from above, top face 4-5-6-7 above it, i.e.
reference corners

    0:(0,0,0) 1:(1,0,0) 2:(1,1,0) 3:(0,1,0)
    4:(0,0,1) 5:(1,0,1) 6:(1,1,1) 7:(0,1,1).
"""

import itertools

import numpy as np

from .rng import uniform, permutation, splitmix64

_CORNERS = np.array(
    [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
     [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.int64)


def _corner_index(c):
    for v in range(8):
        if tuple(_CORNERS[v]) == tuple(c):
            return v
    raise ValueError(c)


def _rotations():
    """The 24 proper rotations of the cube, each as a permutation `perm` of
    local vertices: the rotated element's local vertex v is the original
    element's local vertex perm[v]."""
    out = []
    for axes in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                R[r, axes[r]] = signs[r]
            if round(np.linalg.det(R)) != 1:
                continue
            perm = []
            for v in range(8):
                c = 2 * _CORNERS[v] - 1          # corner in {-1,1}^3
                rc = (R @ c + 1) // 2
                perm.append(_corner_index(rc))
            out.append(tuple(perm))
    assert len(out) == 24
    return np.array(out, dtype=np.int64)


CUBE_ROTATIONS = _rotations()


def hex_lattice(N, perturb=0.0, seed=1, shuffle=False, shuffle_seed=None,
                box=(1.0, 1.0, 1.0)):
    """N^3 hexahedra on the box [0,Lx]x[0,Ly]x[0,Lz] (unit cube by default).

    Returns (coords float64 [nv,3], hex int32 [E,8]).

    perturb: each vertex coordinate d moves by U[-perturb*h_d, perturb*h_d]
      (draw 3*v+d of stream `seed`), except along directions where the vertex
      sits on the boundary (index 0 or N), so boundary vertices move only
      tangentially.
    shuffle: renumber vertices and elements with seeded permutations and give
      each element a seeded random proper rotation of its local vertex order.
    """
    N = int(N)
    if N < 1:
        raise ValueError("N must be >= 1")
    n1 = N + 1
    L = np.asarray(box, dtype=np.float64)
    h = L / N
    k, j, i = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    idx = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)          # [nv,3], x fastest
    coords = idx.astype(np.float64) / N * L
    if perturb > 0.0:
        nv = idx.shape[0]
        d = uniform(seed, 3 * nv, -1.0, 1.0).reshape(nv, 3) * (perturb * h)
        interior = (idx > 0) & (idx < N)
        coords = coords + np.where(interior, d, 0.0)
    ek, ej, ei = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    base = (ei.ravel() + n1 * (ej.ravel() + n1 * ek.ravel())).astype(np.int64)
    off = np.array([0, 1, 1 + n1, n1,
                    n1 * n1, 1 + n1 * n1, 1 + n1 + n1 * n1, n1 + n1 * n1], dtype=np.int64)
    hexes = base[:, None] + off[None, :]
    if shuffle:
        s = seed if shuffle_seed is None else shuffle_seed
        nv = coords.shape[0]
        vperm = permutation(s * 7 + 1, nv)          # new vertex id -> old vertex id
        inv = np.empty(nv, dtype=np.int64)
        inv[vperm] = np.arange(nv)
        coords = coords[vperm]
        hexes = inv[hexes]
        eperm = permutation(s * 7 + 2, hexes.shape[0])
        hexes = hexes[eperm]
        rot = (splitmix64(s * 7 + 3, hexes.shape[0]) % np.uint64(24)).astype(np.int64)
        hexes = np.take_along_axis(hexes, CUBE_ROTATIONS[rot], axis=1)
    return np.ascontiguousarray(coords), np.ascontiguousarray(hexes.astype(np.int32))


def lattice_dofs(N, p):
    """Number of H1 Q_p DOFs on an N^3 lattice: (pN+1)^3."""
    return (p * N + 1) ** 3


def submesh(coords, hexes, keep):
    """Keep the elements listed in `keep` and renumber the vertices they use
    (in order of first use), e.g. to build meshes whose element count is not
    a multiple of a kernel's block size."""
    hexes = np.asarray(hexes, dtype=np.int64)[np.asarray(keep)]
    used, first = np.unique(hexes.ravel(), return_index=True)
    order = used[np.argsort(first, kind="stable")]
    remap = np.full(int(hexes.max()) + 1, -1, dtype=np.int64)
    remap[order] = np.arange(order.size)
    return (np.ascontiguousarray(np.asarray(coords)[order]),
            np.ascontiguousarray(remap[hexes].astype(np.int32)))


def quad_lattice(N, perturb=0.0, seed=1, shuffle=False, shuffle_seed=None):
    """N^2 quadrilaterals on the unit square, local vertex order 0:(0,0)
    1:(1,0) 2:(1,1) 3:(0,1) (counter-clockwise). Returns (coords float64
    [nv,2], quads int32 [E,4]). Perturbation and shuffling as in
    hex_lattice (boundary vertices move only along the boundary; shuffling
    renumbers vertices and elements and rotates each element's vertex list
    cyclically)."""
    N = int(N)
    if N < 1:
        raise ValueError("N must be >= 1")
    n1 = N + 1
    h = 1.0 / N
    j, i = np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij")
    idx = np.stack([i.ravel(), j.ravel()], axis=1)
    coords = idx.astype(np.float64) / N
    if perturb > 0.0:
        nv = idx.shape[0]
        d = uniform(seed, 2 * nv, -1.0, 1.0).reshape(nv, 2) * (perturb * h)
        coords = coords + np.where((idx > 0) & (idx < N), d, 0.0)
    ej, ei = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    base = (ei.ravel() + n1 * ej.ravel()).astype(np.int64)
    quads = base[:, None] + np.array([0, 1, 1 + n1, n1], dtype=np.int64)[None, :]
    if shuffle:
        s = seed if shuffle_seed is None else shuffle_seed
        nv = coords.shape[0]
        vperm = permutation(s * 7 + 1, nv)
        inv = np.empty(nv, dtype=np.int64)
        inv[vperm] = np.arange(nv)
        coords = coords[vperm]
        quads = inv[quads]
        quads = quads[permutation(s * 7 + 2, quads.shape[0])]
        rot = (splitmix64(s * 7 + 3, quads.shape[0]) % np.uint64(4)).astype(np.int64)
        cyc = np.array([[0, 1, 2, 3], [1, 2, 3, 0], [2, 3, 0, 1], [3, 0, 1, 2]], dtype=np.int64)
        quads = np.take_along_axis(quads, cyc[rot], axis=1)
    return np.ascontiguousarray(coords), np.ascontiguousarray(quads.astype(np.int32))


def _bulge(x, amp):
    """Smooth interior displacement of the unit cube / square, zero on its
    boundary: x + amp * prod_d sin(pi x_d) * (1, ..., 1)."""
    s = np.prod(np.sin(np.pi * x), axis=-1, keepdims=True)
    return x + amp * s


def curved_nodes(coords, cells, k, amp=0.05):
    """Per-element nodal coordinates of a curved mesh: every element's
    (k+1)^dim equispaced reference lattice (first index fastest, in the
    element's own local vertex frame), mapped through the element's
    multilinear vertex map and then through a smooth bulge that fixes the
    domain boundary. Neighbours compute identical points on shared faces, so
    the nodal field is continuous. cells: [E,8] hexes (local vertices
    (0,0,0) (1,0,0) (1,1,0) (0,1,0) then z = 1) or [E,4] quads. Returns
    [E, (k+1)^dim, dim]."""
    coords = np.asarray(coords, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    dim = coords.shape[1]
    t = np.arange(k + 1) / k
    if dim == 3:
        c3, c2, c1 = np.meshgrid(t, t, t, indexing="ij")
        xi = np.stack([c1.ravel(), c2.ravel(), c3.ravel()], axis=1)
        corners = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                            [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])
    else:
        c2, c1 = np.meshgrid(t, t, indexing="ij")
        xi = np.stack([c1.ravel(), c2.ravel()], axis=1)
        corners = np.array([[0, 0], [1, 0], [1, 1], [0, 1]])
    W = np.ones((xi.shape[0], corners.shape[0]))
    for v in range(corners.shape[0]):
        for d in range(dim):
            W[:, v] *= np.where(corners[v, d] == 1, xi[:, d], 1.0 - xi[:, d])
    X = np.einsum("kv,evr->ekr", W, coords[cells])
    return _bulge(X, amp)
