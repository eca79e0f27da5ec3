"""Pins for the convection oracle: constants are in its kernel; a constant
velocity on a linear function gives (beta . a) times the mass matrix's row
sums; with a constant velocity the operator is skew-symmetric on interior
DOFs (integration by parts, div beta = 0; exact quadrature of the
polynomial integrand on trilinear meshes); a velocity that is the gradient
of the test function's own coordinates reproduces the stiffness matrix's
action on linear functions; renumbering invariance."""

import numpy as np
import pytest

from fem_inputs import hex_lattice, x_uniform
from oracle import assemble, convection, element


def _const_beta(prob_or_ref, E, b):
    Q3 = prob_or_ref.w.size
    return np.broadcast_to(np.asarray(b, dtype=np.float64), (E, Q3, 3)).copy()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_kernel_linear_and_skew(p):
    c, h = hex_lattice(3, 0.2, seed=4, shuffle=True)
    E = h.shape[0]
    ref = element.Reference(p, p + 2)
    beta = _const_beta(ref, E, [0.7, -0.4, 1.3])
    cp = convection.ConvectionProblem(c, h, p, p + 2, beta)
    C = cp.C
    # constants: C 1 = 0
    assert np.abs(C @ np.ones(cp.ndof)).max() <= 1e-13 * abs(C).max()
    # linear u = a . x: C u = (beta . a) M 1
    tri = assemble.Problem(c, h, p, p + 2)
    X = tri.dof_coords()
    a = np.array([0.3, 1.1, -0.6])
    np.testing.assert_allclose(C @ (X @ a), (beta[0, 0] @ a) * (tri.M @ np.ones(cp.ndof)),
                               atol=1e-13 * abs(C).max())
    # skew-symmetry on interior DOFs
    inter = ~tri.num["boundary_mask"]
    S = (C + C.T).toarray()[np.ix_(inter, inter)]
    assert np.abs(S).max() <= 1e-13 * abs(C).max()
    assert abs(C).max() > 1e-3


def test_variable_velocity_against_direct_quadrature():
    """beta(x) = (x1, x2^2, x0 x1) at the points: C u for u = x0 + 2 x2 equals
    sum_q w detJ phi_i (beta . (1, 0, 2)) (the same sum with grad u known)."""
    p = 2
    c, h = hex_lattice(2, 0.15, seed=8)
    ref = element.Reference(p, p + 2)
    x, _, det, _ = element.geometry(ref, c[h.astype(np.int64)])
    beta = np.stack([x[..., 1], x[..., 2] ** 2, x[..., 0] * x[..., 1]], -1)
    cp = convection.ConvectionProblem(c, h, p, p + 2, beta)
    tri = assemble.Problem(c, h, p, p + 2)
    X = tri.dof_coords()
    u = X[:, 0] + 2.0 * X[:, 2]
    be = np.einsum("qi,eq->ei", ref.phi, ref.w[None, :] * det * (beta[..., 0] + 2.0 * beta[..., 2]))
    ref_b = np.zeros(cp.ndof)
    np.add.at(ref_b, cp.e2l.ravel(), be.ravel())
    np.testing.assert_allclose(cp.apply(u), ref_b, atol=1e-13 * np.abs(ref_b).max())


def test_invariance_under_renumbering():
    p = 2
    c0, h0 = hex_lattice(2, 0.1, seed=7)
    c1, h1 = hex_lattice(2, 0.1, seed=7, shuffle=True, shuffle_seed=11)
    ref = element.Reference(p, p + 2)
    P = []
    for c, h in ((c0, h0), (c1, h1)):
        x, _, _, _ = element.geometry(ref, c[h.astype(np.int64)])
        beta = np.stack([np.sin(x[..., 1]), x[..., 0], 1.0 + x[..., 2]], -1)
        P.append((convection.ConvectionProblem(c, h, p, p + 2, beta), assemble.Problem(c, h, p, p + 2)))
    X0, X1 = P[0][1].dof_coords(), P[1][1].dof_coords()
    key = lambda X: np.lexsort(np.round(X, 11).T[::-1])
    o0, o1 = key(X0), key(X1)
    perm = np.empty(X0.shape[0], dtype=np.int64)
    perm[o0] = o1
    np.testing.assert_allclose(P[1][0].C.toarray()[np.ix_(perm, perm)], P[0][0].C.toarray(), atol=1e-12)
