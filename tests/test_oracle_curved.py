"""Pins for the curved (nodal) geometry oracle: order-k nodes that describe
a trilinear map reproduce the trilinear oracle exactly; a polynomial map's
volume matches its exact integral; the isoparametric patch test holds on a
genuinely curved mesh (linear functions lie in the space when p >= k);
renumbering and element rotation leave the operator unchanged."""

import numpy as np
import pytest
import sympy as sy

from fem_inputs import curved_nodes, hex_lattice, lognormal
from oracle import assemble, curved, lagrange, numbering, rules


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_trilinear_as_nodes(k, p):
    c, h = hex_lattice(2, 0.2, seed=3, shuffle=True)
    kap = lognormal(4, h.shape[0])
    tri = assemble.Problem(c, h, p, p + 2, kappa=kap, rho=kap)
    Xn = curved.nodes_from_corners(c[h.astype(np.int64)], k)
    if k == 1:  # the order-1 lattice (x fastest) visits the corners 0, 1, 3, 2, 4, 5, 7, 6
        np.testing.assert_array_equal(Xn, c[h.astype(np.int64)][:, [0, 1, 3, 2, 4, 5, 7, 6]])
    cp = curved.CurvedProblem(h, Xn, k, p, p + 2, kappa=kap, rho=kap)
    for kind in ("diffusion", "mass"):
        A, B = cp.matrix(kind).toarray(), tri.matrix(kind).toarray()
        assert np.abs(A - B).max() <= 1e-13 * np.abs(B).max()
    np.testing.assert_allclose(cp.dof_coords(), tri.dof_coords(), atol=1e-14)
    np.testing.assert_allclose(cp.qpoint_coords(), tri.qpoint_coords(), atol=1e-14)


def test_volume_of_polynomial_map():
    """Single element, Phi(xi) = (x + a x(1-x) y, y + b y(1-y) z^2, z + c x y z):
    degree <= 2 per variable, so order-2 GLL nodes reproduce it exactly and
    the mass matrix's total equals int det(grad Phi) over the unit cube."""
    a, b, cc = 0.3, -0.25, 0.2
    xs, ys, zs = sy.symbols("x y z")
    Phi = sy.Matrix([xs + a * xs * (1 - xs) * ys, ys + b * ys * (1 - ys) * zs ** 2, zs + cc * xs * ys * zs])
    Jac = Phi.jacobian([xs, ys, zs])
    vol = float(sy.integrate(Jac.det(), (xs, 0, 1), (ys, 0, 1), (zs, 0, 1)))
    xi = rules.gll_nodes(2)[numbering.lattice(2)]
    f = sy.lambdify((xs, ys, zs), Phi, "numpy")
    Xn = np.stack([np.asarray(f(*pt), dtype=np.float64).ravel() for pt in xi])[None]
    hexes = np.arange(8)[None]
    cp = curved.CurvedProblem(hexes, Xn, 2, 2, 6)
    one = np.ones(cp.ndof)
    assert one @ (cp.M @ one) == pytest.approx(vol, abs=1e-13)
    assert abs(vol - 1.0) > 1e-3          # the map is not volume preserving


@pytest.mark.parametrize("k,p", [(2, 2), (2, 3), (3, 3)])
def test_isoparametric_patch_test(k, p):
    c, h = hex_lattice(3, 0.1, seed=5)
    Xg = curved_nodes(c, h, k, amp=0.06)
    # reinterpret the equispaced points as the values at the GLL lattice:
    # any nodal field is a valid geometry; linear functions of x are in the
    # space because x itself is a Q_k function of the reference coordinates
    cp = curved.CurvedProblem(h, Xg, k, p, p + 2)   # kappa = 1: a jump in kappa breaks the patch test
    X = cp.dof_coords()
    bnd = cp.num["boundary_mask"]
    Kd = cp.K
    for g in (np.array([1.0, 0.0, 0.0]), np.array([0.3, -1.1, 0.7])):
        r = Kd @ (X @ g + 0.25)
        assert np.abs(r[~bnd]).max() <= 1e-11 * abs(Kd).max()
    # constants are in the kernel; the boundary nodes stay on the cube's faces,
    # so the domain is still the unit cube: volume 1 (det J is a polynomial
    # the q = p + 2 rule integrates exactly); and the mesh is genuinely
    # curved (its mass matrix differs from the trilinear one)
    assert np.abs(Kd @ np.ones(cp.ndof)).max() <= 1e-12 * abs(Kd).max()
    one = np.ones(cp.ndof)
    assert one @ (cp.M @ one) == pytest.approx(1.0, abs=1e-12)
    tri = assemble.Problem(c, h, p, p + 2)
    assert np.abs(cp.M.toarray() - tri.M.toarray()).max() > 1e-6


def test_invariance_under_renumbering():
    k, p = 2, 2
    c0, h0 = hex_lattice(2, 0.1, seed=7)
    c1, h1 = hex_lattice(2, 0.1, seed=7, shuffle=True, shuffle_seed=11)
    P0 = curved.CurvedProblem(h0, curved_nodes(c0, h0, k), k, p, p + 2)
    P1 = curved.CurvedProblem(h1, curved_nodes(c1, h1, k), k, p, p + 2)
    X0, X1 = P0.dof_coords(), P1.dof_coords()
    key = lambda X: np.lexsort(np.round(X, 11).T[::-1])
    o0, o1 = key(X0), key(X1)
    np.testing.assert_allclose(X0[o0], X1[o1], atol=1e-12)
    perm = np.empty(P0.ndof, dtype=np.int64)
    perm[o0] = o1
    np.testing.assert_allclose(P1.K.toarray()[np.ix_(perm, perm)], P0.K.toarray(), atol=1e-11)


# ---------------------------------------------------------------- 2D ----
from fem_inputs import quad_lattice
from oracle import twod


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_bilinear_as_nodes_2d(k, p):
    c, q = quad_lattice(3, 0.2, seed=13, shuffle=True)
    kap = lognormal(14, q.shape[0])
    bil = twod.Problem2(c, q, p, p + 2, kappa=kap, rho=kap)
    Xn = curved.nodes_from_corners2(c[q.astype(np.int64)], k)
    if k == 1:  # the order-1 lattice (x fastest) visits the corners 0, 1, 3, 2
        np.testing.assert_array_equal(Xn, c[q.astype(np.int64)][:, [0, 1, 3, 2]])
    cp = curved.CurvedProblem2(q, Xn, k, p, p + 2, kappa=kap, rho=kap, nv=c.shape[0])
    for kind in ("diffusion", "mass"):
        A, B = cp.matrix(kind).toarray(), bil.matrix(kind).toarray()
        assert np.abs(A - B).max() <= 1e-13 * np.abs(B).max()
    np.testing.assert_allclose(cp.dof_coords(), bil.dof_coords(), atol=1e-14)
    np.testing.assert_allclose(cp.qpoint_coords(), bil.qpoint_coords(), atol=1e-14)


def test_area_of_polynomial_map_2d():
    """Single element, Phi(x, y) = (x (1 + a y^2), y (1 + b x^2)): degree
    <= 2 per variable, so order-2 GLL nodes reproduce it exactly and the mass
    matrix's total equals int det(grad Phi) over the unit square (the right
    and top edges are curved, so the area is not 1)."""
    a, b = 0.35, -0.3
    xs, ys = sy.symbols("x y")
    Phi = sy.Matrix([xs * (1 + a * ys ** 2), ys * (1 + b * xs ** 2)])
    area = float(sy.integrate(Phi.jacobian([xs, ys]).det(), (xs, 0, 1), (ys, 0, 1)))
    xi = curved.lattice_nodes2(2)
    f = sy.lambdify((xs, ys), Phi, "numpy")
    Xn = np.stack([np.asarray(f(*pt), dtype=np.float64).ravel() for pt in xi])[None]
    cp = curved.CurvedProblem2(np.arange(4)[None], Xn, 2, 2, 5)
    one = np.ones(cp.ndof)
    assert one @ (cp.M @ one) == pytest.approx(area, abs=1e-14)
    assert abs(area - 1.0) > 1e-3          # the map is not area preserving
    # and the stiffness matrix annihilates constants
    assert np.abs(cp.K @ one).max() <= 1e-13 * abs(cp.K).max()


@pytest.mark.parametrize("k,p", [(2, 2), (2, 3), (3, 3), (4, 5)])
def test_isoparametric_patch_test_2d(k, p):
    c, q = quad_lattice(4, 0.1, seed=15)
    Xg = curved_nodes(c, q, k, amp=0.06)
    cp = curved.CurvedProblem2(q, Xg, k, p, p + 2, nv=c.shape[0])
    X = cp.dof_coords()
    bnd = cp.num["boundary_mask"]
    Kd = cp.K
    for g in (np.array([1.0, 0.0]), np.array([0.3, -1.1])):
        r = Kd @ (X @ g + 0.25)
        assert np.abs(r[~bnd]).max() <= 1e-11 * abs(Kd).max()
    one = np.ones(cp.ndof)
    assert np.abs(Kd @ one).max() <= 1e-12 * abs(Kd).max()
    assert one @ (cp.M @ one) == pytest.approx(1.0, abs=1e-12)   # the boundary stays on the unit square
    bil = twod.Problem2(c, q, p, p + 2)
    assert np.abs(cp.M.toarray() - bil.M.toarray()).max() > 1e-6


def test_invariance_under_renumbering_2d():
    k, p = 3, 2
    c0, q0 = quad_lattice(3, 0.1, seed=17)
    c1, q1 = quad_lattice(3, 0.1, seed=17, shuffle=True, shuffle_seed=19)
    P0 = curved.CurvedProblem2(q0, curved_nodes(c0, q0, k), k, p, p + 2, nv=c0.shape[0])
    P1 = curved.CurvedProblem2(q1, curved_nodes(c1, q1, k), k, p, p + 2, nv=c1.shape[0])
    X0, X1 = P0.dof_coords(), P1.dof_coords()
    key = lambda X: np.lexsort(np.round(X, 11).T[::-1])
    o0, o1 = key(X0), key(X1)
    np.testing.assert_allclose(X0[o0], X1[o1], atol=1e-12)
    perm = np.empty(P0.ndof, dtype=np.int64)
    perm[o0] = o1
    np.testing.assert_allclose(P1.K.toarray()[np.ix_(perm, perm)], P0.K.toarray(), atol=1e-11)
