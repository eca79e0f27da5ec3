"""The library's host code (mesh ingest, topology, DOF numbering, inverse
map, boundary DOFs; csrc/fem_host.cpp and fem_basis.cpp) on CPU: the sources
are compiled against a test-only stand-in for the CUDA runtime
(tests/host_stub: device memory is host memory) and called through the same
C ABI. The element->DOF table and the boundary DOF list must equal the
oracle's, built independently from entity keys (bit for bit), for 3D and
2D meshes, shuffled vertex orders, several orders on one mesh (the shared
topology), and meshes large enough for the multithreaded fill."""

import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from fem_inputs import hex_lattice, quad_lattice
from oracle import numbering, twod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1911_09220_gb300", "csrc")


@pytest.fixture(scope="module")
def hostlib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("hostlib") / "libfem_host_test.so")
    # -Bsymbolic: the library's calls bind to its own definitions even when
    # the real libfem.so / libcudart were loaded globally by another test
    cmd = ["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-pthread", "-Wl,-Bsymbolic",
           "-I", os.path.join(ROOT, "tests", "host_stub"),
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, os.path.join(CSRC, "fem_host.cpp"),
           os.path.join(CSRC, "fem_basis.cpp"), os.path.join(ROOT, "tests", "host_stub", "stub.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = C.CDLL(out, mode=C.RTLD_LOCAL)
    P, I64 = C.c_void_p, C.c_int64
    for name, res, args in [("fem_mesh_create", C.c_int, [P, I64, P, I64, C.POINTER(P)]),
                            ("fem_mesh2d_create", C.c_int, [P, I64, P, I64, C.POINTER(P)]),
                            ("fem_space_create", C.c_int, [P, C.c_int, C.POINTER(P)]),
                            ("fem_space_info", C.c_int, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64),
                                                         C.POINTER(C.c_int)]),
                            ("fem_space_element_dofs", C.c_int, [P, P]),
                            ("fem_space_boundary_dofs", C.c_int, [P, P]),
                            ("fem_space_destroy", None, [P]), ("fem_mesh_destroy", None, [P]),
                            ("fem_last_error", C.c_char_p, [])]:
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    return L


def _mesh(L, coords, cells, dim):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    m = C.c_void_p()
    create = L.fem_mesh_create if dim == 3 else L.fem_mesh2d_create
    assert create(coords.ctypes.data, coords.shape[0], cells.ctypes.data, cells.shape[0], C.byref(m)) == 0, \
        L.fem_last_error()
    return m


def _space(L, m, p):
    s = C.c_void_p()
    assert L.fem_space_create(m, p, C.byref(s)) == 0, L.fem_last_error()
    ndof, nbdr, ne = C.c_int64(), C.c_int64(), C.c_int64()
    pp = C.c_int()
    assert L.fem_space_info(s, C.byref(ndof), C.byref(nbdr), C.byref(ne), C.byref(pp)) == 0
    return s, ndof.value, nbdr.value, ne.value


def _tables(L, s, ne, nd, nbdr):
    e2l = np.empty((ne, nd), dtype=np.int32)
    bdr = np.empty(nbdr, dtype=np.int32)
    assert L.fem_space_element_dofs(s, e2l.ctypes.data) == 0
    assert L.fem_space_boundary_dofs(s, bdr.ctypes.data) == 0
    return e2l, bdr


@pytest.mark.parametrize("N,shuffle", [(3, False), (3, True), (20, True)])
def test_3d_numbering_matches_oracle(hostlib, N, shuffle):
    L = hostlib
    c, h = hex_lattice(N, 0.1, seed=2, shuffle=shuffle)
    m = _mesh(L, c, h, 3)
    orders = [4, 2, 1, 3] if N <= 3 else [2, 1]
    for p in orders:                       # several spaces on one mesh: shared topology
        s, ndof, nbdr, ne = _space(L, m, p)
        e2l, bdr = _tables(L, s, ne, (p + 1) ** 3, nbdr)
        num = numbering.build(h, p, nv=c.shape[0])
        assert ndof == num["ndof"]
        assert np.array_equal(e2l, num["e2l"])
        assert np.array_equal(bdr, np.asarray(num["boundary_dofs"], dtype=np.int32))
        L.fem_space_destroy(s)
    L.fem_mesh_destroy(m)


@pytest.mark.parametrize("p", [1, 2, 5])
def test_2d_numbering_matches_oracle(hostlib, p):
    L = hostlib
    c, q = quad_lattice(5, 0.1, seed=3, shuffle=True)
    m = _mesh(L, c, q, 2)
    s = C.c_void_p()
    assert L.fem_space_create(m, p, C.byref(s)) == 0
    ndof, nbdr, ne = C.c_int64(), C.c_int64(), C.c_int64()
    pp = C.c_int()
    L.fem_space_info(s, C.byref(ndof), C.byref(nbdr), C.byref(ne), C.byref(pp))
    e2l, bdr = _tables(L, s, ne.value, (p + 1) ** 2, nbdr.value)
    num = twod.numbering2(q, p, nv=c.shape[0])
    assert ndof.value == num["ndof"]
    assert np.array_equal(e2l, num["e2l"])
    assert np.array_equal(bdr, np.asarray(num["boundary_dofs"], dtype=np.int32))
    L.fem_space_destroy(s)
    L.fem_mesh_destroy(m)


def test_mesh_errors(hostlib):
    L = hostlib
    c, h = hex_lattice(2, 0.0, seed=1)
    bad = h.copy()
    bad[0, 1] = bad[0, 0]                  # repeated vertex
    m = C.c_void_p()
    coords = np.ascontiguousarray(c)
    assert L.fem_mesh_create(coords.ctypes.data, c.shape[0], bad.ctypes.data, bad.shape[0], C.byref(m)) == 1
    assert len(L.fem_last_error()) > 0
    m = _mesh(L, c, h, 3)
    s = C.c_void_p()
    assert L.fem_space_create(m, 0, C.byref(s)) == 1
    assert L.fem_space_create(m, 9, C.byref(s)) == 7
    L.fem_mesh_destroy(m)


@pytest.mark.parametrize("seed", range(8))
def test_numbering_over_random_orderings(hostlib, seed):
    """Random vertex and element numberings with random proper rotations of
    every element's vertex list (fem_inputs' shuffle): the library's table
    equals the oracle's for p = 3."""
    L = hostlib
    c, h = hex_lattice(3, 0.12, seed=40 + seed, shuffle=True, shuffle_seed=500 + seed)
    m = _mesh(L, c, h, 3)
    s, ndof, nbdr, ne = _space(L, m, 3)
    e2l, bdr = _tables(L, s, ne, 64, nbdr)
    num = numbering.build(h, 3, nv=c.shape[0])
    assert np.array_equal(e2l, num["e2l"]) and np.array_equal(bdr, np.asarray(num["boundary_dofs"], np.int32))
    L.fem_space_destroy(s)
    L.fem_mesh_destroy(m)


def test_malformed_meshes_are_rejected(hostlib):
    L = hostlib
    c, h = hex_lattice(2, 0.0, seed=1)
    coords = np.ascontiguousarray(c)
    m = C.c_void_p()

    def create(cc, hh, nv=None, ne=None):
        cc = np.ascontiguousarray(cc, dtype=np.float64)
        hh = np.ascontiguousarray(hh, dtype=np.int32)
        return L.fem_mesh_create(cc.ctypes.data, cc.shape[0] if nv is None else nv, hh.ctypes.data,
                                 hh.shape[0] if ne is None else ne, C.byref(m))

    assert create(c, h, ne=0) == 1                       # no elements
    assert create(c, h, nv=0) == 1                       # no vertices
    bad = h.copy()
    bad[3, 5] = c.shape[0]                               # index out of range
    assert create(c, bad) == 1
    bad = h.copy()
    bad[2, 0] = -1                                       # negative index
    assert create(c, bad) == 1
    extra = np.vstack([c, [[5.0, 5.0, 5.0]]])            # a vertex no element uses
    assert create(extra, h) == 1
    assert L.fem_mesh_create(None, c.shape[0], h.ctypes.data, h.shape[0], C.byref(m)) == 1
    assert create(c, h) == 0                             # the valid mesh still builds
    L.fem_mesh_destroy(m)


@pytest.mark.parametrize("pf,pc", [(2, 1), (4, 2), (5, 2), (8, 4)])
def test_multigrid_coarse_essential_rule(hostlib, pf, pc):
    """The library's p-multigrid coarse essential rule (coarse DOF essential
    iff every fine DOF of its mesh entity is) against the oracle's, for the
    whole boundary, one face and random masks."""
    from oracle import multigrid as omg
    L = hostlib
    f = L.test_coarse_essential
    f.restype, f.argtypes = C.c_int64, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    c, h = hex_lattice(3, 0.1, seed=9, shuffle=True)
    m = _mesh(L, c, h, 3)
    sf, nf, nbf, ne = _space(L, m, pf)
    sc, nc, nbc, _ = _space(L, m, pc)
    e2lf, bdrf = _tables(L, sf, ne, (pf + 1) ** 3, nbf)
    e2lc, _ = _tables(L, sc, ne, (pc + 1) ** 3, nbc)
    from oracle import assemble
    X = assemble.Problem(c, h, pf, pf + 2).dof_coords()
    rng = np.random.default_rng(pf * 10 + pc)
    masks = [np.isin(np.arange(nf), bdrf), np.abs(X[:, 0]) < 1e-12, rng.random(nf) < 0.5, rng.random(nf) < 0.95]
    for mask in masks:
        mk = np.ascontiguousarray(mask.astype(np.uint8))
        out = np.empty(nc, dtype=np.int32)
        cnt = f(sf, mk.ctypes.data, sc, out.ctypes.data)
        ref = np.nonzero(omg.coarse_essential(e2lf, pf, mask, e2lc, pc, nc))[0]
        assert np.array_equal(out[:cnt], ref.astype(np.int32))
    L.fem_space_destroy(sf)
    L.fem_space_destroy(sc)
    L.fem_mesh_destroy(m)


def test_set_nodes_validation(hostlib):
    L = hostlib
    f = L.fem_mesh_set_nodes
    f.restype, f.argtypes = C.c_int, [C.c_void_p, C.c_int, C.c_void_p]
    c, h = hex_lattice(2, 0.1, seed=4)
    m = _mesh(L, c, h, 3)
    E = h.shape[0]
    for k in (1, 2, 8):
        nodes = np.zeros((E, (k + 1) ** 3, 3))
        assert f(m, k, nodes.ctypes.data) == 0
    assert f(m, 0, None) == 0                           # back to the vertex geometry
    assert f(m, 9, np.zeros((E, 1000, 3)).ctypes.data) == 1
    assert f(m, -1, None) == 1
    assert f(m, 2, None) == 1
    bad = np.zeros((E, 27, 3))
    bad[3, 5, 1] = np.nan
    assert f(m, 2, bad.ctypes.data) == 1
    bad[3, 5, 1] = np.inf
    assert f(m, 2, bad.ctypes.data) == 1
    # spaces on a mesh with nodes: the numbering does not change
    good = np.zeros((E, 27, 3))
    assert f(m, 2, good.ctypes.data) == 0
    s, ndof, nbdr, ne = _space(L, m, 2)
    e2l, _ = _tables(L, s, ne, 27, nbdr)
    assert np.array_equal(e2l, numbering.build(h, 2, nv=c.shape[0])["e2l"])
    L.fem_space_destroy(s)
    L.fem_mesh_destroy(m)
    # quadrilateral meshes take [ne][(k+1)^2][2] nodes: exactly that many
    # values are read and checked (a non-finite last value is caught)
    cq, q = quad_lattice(2, 0.0, seed=1)
    m2 = _mesh(L, cq, q, 2)
    E2 = q.shape[0]
    g2 = np.zeros((E2, 9, 2))
    assert f(m2, 2, g2.ctypes.data) == 0
    g2[-1, -1, -1] = np.nan
    assert f(m2, 2, g2.ctypes.data) == 1
    assert f(m2, 0, None) == 0
    L.fem_mesh_destroy(m2)
