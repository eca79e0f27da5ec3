"""Pins for the elasticity oracle: the six rigid-body modes (translations and
infinitesimal rotations, exactly representable on trilinear meshes) are in
the kernel on every row; a linear displacement (constant strain) passes the
patch test on interior rows; the component-diagonal blocks sum to
(lambda + 4 mu) times the scalar stiffness matrix; symmetry and positive
semi-definiteness; renumbering invariance."""

import numpy as np
import pytest

from fem_inputs import hex_lattice, lognormal
from oracle import assemble, elasticity


def _vec(X, f):
    """Stack f(X) [ndof,3] component-major."""
    return np.concatenate([f(X)[:, c] for c in range(3)])


@pytest.mark.parametrize("p", [1, 2, 3])
def test_rigid_modes_patch_and_trace(p):
    c, h = hex_lattice(3, 0.2, seed=4, shuffle=True)
    E = h.shape[0]
    lam, mu = lognormal(1, E), lognormal(2, E)
    ep = elasticity.ElasticityProblem(c, h, p, p + 2, lam, mu)
    tri = assemble.Problem(c, h, p, p + 2)
    X = tri.dof_coords()
    K = ep.K
    kmax = abs(K).max()
    modes = [lambda X, d=d: np.eye(3)[d][None, :] + 0 * X for d in range(3)]
    for axis in range(3):
        w = np.eye(3)[axis]
        modes.append(lambda X, w=w: np.cross(w[None, :], X))
    for f in modes:
        assert np.abs(K @ _vec(X, f)).max() <= 1e-12 * kmax
    # constant strain with constant coefficients: interior rows vanish
    ep1 = elasticity.ElasticityProblem(c, h, p, p + 2, np.full(E, 1.7), np.full(E, 0.6))
    A = np.array([[0.3, -0.2, 0.5], [0.1, 0.8, -0.4], [0.7, 0.2, -0.6]])
    u = _vec(X, lambda X: X @ A.T)
    inter = np.tile(~tri.num["boundary_mask"], 3)
    r = ep1.K @ u
    assert np.abs(r[inter]).max() <= 1e-12 * abs(ep1.K).max()
    assert np.abs(r).max() > 1e-6        # boundary rows carry the traction
    # component trace identity
    n = ep.ndof
    tr = sum(K[cc * n:(cc + 1) * n, cc * n:(cc + 1) * n] for cc in range(3))
    Lk = assemble.Problem(c, h, p, p + 2, kappa=lam + 4 * mu).K
    assert abs(tr - Lk).max() <= 1e-12 * kmax
    # symmetry, positive semi-definiteness
    assert abs(K - K.T).max() <= 1e-13 * kmax
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.uniform(-1, 1, 3 * n)
        assert v @ (K @ v) > 0


def test_invariance_under_renumbering():
    p = 2
    c0, h0 = hex_lattice(2, 0.1, seed=7)
    c1, h1 = hex_lattice(2, 0.1, seed=7, shuffle=True, shuffle_seed=11)
    E = h0.shape[0]
    P0 = elasticity.ElasticityProblem(c0, h0, p, p + 2, np.full(E, 2.0), np.full(E, 0.5))
    P1 = elasticity.ElasticityProblem(c1, h1, p, p + 2, np.full(E, 2.0), np.full(E, 0.5))
    X0 = assemble.Problem(c0, h0, p, p + 2).dof_coords()
    X1 = assemble.Problem(c1, h1, p, p + 2).dof_coords()
    key = lambda X: np.lexsort(np.round(X, 11).T[::-1])
    o0, o1 = key(X0), key(X1)
    perm = np.empty(X0.shape[0], dtype=np.int64)
    perm[o0] = o1
    n = X0.shape[0]
    vperm = np.concatenate([perm + cc * n for cc in range(3)])
    np.testing.assert_allclose(P1.K.toarray()[np.ix_(vperm, vperm)], P0.K.toarray(), atol=1e-11)


@pytest.mark.parametrize("k", [1, 2])
def test_nodal_geometry_of_a_trilinear_mesh(k):
    """The order-k nodal geometry that writes the trilinear map as a grid
    function gives the trilinear operator (same J at every point)."""
    from oracle import curved
    c, h = hex_lattice(2, 0.2, seed=9, shuffle=True)
    E = h.shape[0]
    lam, mu = lognormal(5, E), lognormal(6, E)
    P0 = elasticity.ElasticityProblem(c, h, 2, 4, lam, mu)
    Xn = curved.nodes_from_corners(c[h.astype(np.int64)], k)
    P1 = elasticity.ElasticityProblem(c, h, 2, 4, lam, mu, Xn=Xn, k=k)
    assert abs(P0.K - P1.K).max() <= 1e-12 * abs(P0.K).max()


@pytest.mark.parametrize("p", [2, 3])
def test_reproduces_a_quadratic_solution(p):
    """Affine mesh, constant lambda and mu: a quadratic displacement u lies
    in the space, the body force f = -div sigma(u) = -((lambda + mu)
    grad div u + mu lap u) is constant, so the discrete solution with
    u on the boundary is u's interpolant itself (to rounding). The force is
    derived symbolically (sympy), independently of the oracle's matrices."""
    sympy = pytest.importorskip("sympy")
    from oracle import solve as osolve
    c, h = hex_lattice(2, 0.0, seed=1, shuffle=True)
    A = np.array([[1.2, 0.3, -0.4], [0.2, 0.9, 0.1], [-0.1, 0.25, 1.1]])    # affine map of the unit cube
    c = c @ A.T + np.array([0.3, -0.2, 0.1])
    E = h.shape[0]
    lam_v, mu_v = 1.7, 0.6
    x, y, z = sympy.symbols("x y z")
    X = (x, y, z)
    u = [x * y - 0.5 * z ** 2 + 0.3 * x, 0.7 * x ** 2 + y * z - 0.2 * y, -0.4 * x * z + 0.9 * y ** 2 + z]
    div = sum(sympy.diff(u[i], X[i]) for i in range(3))
    f = [-((lam_v + mu_v) * sympy.diff(div, X[i]) + mu_v * sum(sympy.diff(u[i], X[j], 2) for j in range(3)))
         for i in range(3)]
    assert all(sympy.simplify(fi).is_number for fi in f)
    fvals = [float(fi) for fi in f]
    ep = elasticity.ElasticityProblem(c, h, p, p + 2, np.full(E, lam_v), np.full(E, mu_v))
    sc = assemble.Problem(c, h, p, p + 2)
    Xd = sc.dof_coords()
    ufun = [sympy.lambdify(X, ui, "numpy") for ui in u]
    uvec = np.concatenate([np.broadcast_to(ufun[k](Xd[:, 0], Xd[:, 1], Xd[:, 2]), (sc.ndof,)) for k in range(3)])
    b = np.concatenate([sc.load(lambda Y, v=fvals[k]: np.full(Y.shape[:-1], v)) for k in range(3)])
    n = sc.ndof
    bd = sc.num["boundary_dofs"]
    ess = np.concatenate([bd + k * n for k in range(3)])
    bc = osolve.constrain_rhs(ep.K, b, ess, uvec[ess])
    Ac = osolve.constrain(ep.K, ess)
    uh = osolve.cholesky_solve(Ac, bc)
    assert np.abs(uh - uvec).max() <= 1e-11 * np.abs(uvec).max()


@pytest.mark.parametrize("p", [1, 2])
def test_convergence_smooth_solution(p):
    """Smooth manufactured displacement on an affinely mapped cube, constant
    lambda and mu, Dirichlet data from u: the nodal error of the discrete
    solution falls at about the rate h^(p+1) under uniform refinement."""
    sympy = pytest.importorskip("sympy")
    from oracle import solve as osolve
    lam_v, mu_v = 2.0, 0.7
    x, y, z = sympy.symbols("x y z")
    X = (x, y, z)
    u = [sympy.sin(x + 0.5 * y) * sympy.cos(z), sympy.exp(0.3 * x) * sympy.sin(y - z), x * y * z + sympy.cos(x - y)]
    div = sum(sympy.diff(u[i], X[i]) for i in range(3))
    f = [-((lam_v + mu_v) * sympy.diff(div, X[i]) + mu_v * sum(sympy.diff(u[i], X[j], 2) for j in range(3)))
         for i in range(3)]
    uf = [sympy.lambdify(X, ui, "numpy") for ui in u]
    ff = [sympy.lambdify(X, fi, "numpy") for fi in f]
    A = np.array([[1.0, 0.2, 0.0], [0.0, 1.1, -0.1], [0.1, 0.0, 0.9]])
    errs = []
    for N in (2, 4):
        c, h = hex_lattice(N, 0.0, seed=1)
        c = c @ A.T
        E = h.shape[0]
        ep = elasticity.ElasticityProblem(c, h, p, p + 2, np.full(E, lam_v), np.full(E, mu_v))
        sc = assemble.Problem(c, h, p, p + 2)
        Xd = sc.dof_coords()
        n = sc.ndof
        uex = np.concatenate([np.broadcast_to(uf[k](Xd[:, 0], Xd[:, 1], Xd[:, 2]), (n,)) for k in range(3)])
        b = np.concatenate([sc.load(lambda Y, k=k: np.broadcast_to(ff[k](Y[..., 0], Y[..., 1], Y[..., 2]),
                                                                   Y.shape[:-1])) for k in range(3)])
        bd = sc.num["boundary_dofs"]
        ess = np.concatenate([bd + k * n for k in range(3)])
        uh = osolve.cholesky_solve(osolve.constrain(ep.K, ess), osolve.constrain_rhs(ep.K, b, ess, uex[ess]))
        errs.append(np.abs(uh - uex).max())
    rate = np.log2(errs[0] / errs[1])
    assert rate > p + 0.6, (errs, rate)


def test_sampled_apply_matches_assembled():
    from fem_inputs import x_uniform
    c, h = hex_lattice(3, 0.15, seed=31, shuffle=True)
    E = h.shape[0]
    lam, mu = lognormal(32, E), lognormal(33, E)
    ep = elasticity.ElasticityProblem(c, h, 2, 4, lam, mu)
    x = x_uniform(34, 3 * ep.ndof)
    rows = np.unique(np.random.default_rng(3).integers(0, 3 * ep.ndof, 40))
    ref = (ep.K @ x)[rows]
    got = elasticity.sampled_apply(c, h, ep.e2l, 2, 4, lam, mu, x, rows)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ep.K @ x).max()
