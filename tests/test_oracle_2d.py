"""Pins for the 2D (quadrilateral) oracle: closed-form Q1 element matrices
and stencil, Kronecker structure, patch test, area, renumbering/rotation
invariance and a hand-derived numbering."""

import numpy as np
import pytest

from fem_inputs import quad_lattice, lognormal
from oracle import twod


def test_q1_square_closed_forms():
    for h in (1.0, 0.25):
        c, qd = quad_lattice(1, 0.0)
        c = c * h
        P = twod.Problem2(c, qd, 1, 2)
        e2l = P.e2l[0]
        K, M = P.K.toarray(), P.M.toarray()
        # lexicographic local order (0,0),(1,0),(0,1),(1,1); 2D stiffness is h-independent
        np.testing.assert_allclose(K[e2l[0], e2l], np.array([4, -1, -1, -2]) / 6.0, atol=1e-15)
        np.testing.assert_allclose(M[e2l[0], e2l], h * h * np.array([4, 2, 2, 1]) / 36.0, atol=1e-16)


def test_q1_nine_point_stencil():
    N = 3
    c, qd = quad_lattice(N, 0.0)
    K = twod.Problem2(c, qd, 1, 3).K.toarray()
    vid = lambda i, j: i + (N + 1) * j
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            expect = 8.0 / 3.0 if di == dj == 0 else -1.0 / 3.0
            assert K[vid(1, 1), vid(1 + di, 1 + dj)] == pytest.approx(expect, abs=1e-15)


@pytest.mark.parametrize("p", [1, 2, 4, 8])
def test_kronecker_structure(p):
    h = 0.5
    c, qd = quad_lattice(1, 0.0)
    c = c * h
    ref = twod.Reference2(p, p + 2)
    X = c[qd.astype(np.int64)]
    Ke = twod.stiffness2(ref, X, [1.0])[0]
    Me = twod.mass2(ref, X, [1.0])[0]
    w = ref.qwts
    K1 = ref.G.T @ np.diag(w) @ ref.G
    M1 = ref.B.T @ np.diag(w) @ ref.B
    np.testing.assert_allclose(Ke, np.kron(M1, K1) + np.kron(K1, M1), atol=1e-12 * np.abs(Ke).max())
    np.testing.assert_allclose(Me, h * h * np.kron(M1, M1), atol=1e-14 * np.abs(Me).max())


@pytest.mark.parametrize("p,shuffle", [(1, False), (2, True), (4, True), (8, False)])
def test_patch_area_symmetry(p, shuffle):
    c, qd = quad_lattice(4, 0.2, seed=3, shuffle=shuffle)
    P = twod.Problem2(c, qd, p, p + 2)
    K, M = P.K, P.M
    one = np.ones(P.ndof)
    assert np.abs(K @ one).max() < 1e-12 * abs(K).max()
    assert one @ (M @ one) == pytest.approx(1.0, abs=1e-13)
    X = P.dof_coords()
    interior = ~P.num["boundary_mask"]
    for g in (np.array([1.0, 0.0]), np.array([0.4, -1.3])):
        r = K @ (X @ g)
        assert np.abs(r[interior]).max() < 1e-12 * abs(K).max()
    xv = np.random.default_rng(0).uniform(-1, 1, P.ndof)
    yv = np.random.default_rng(1).uniform(-1, 1, P.ndof)
    assert abs(xv @ (K @ yv) - yv @ (K @ xv)) < 1e-12 * abs(K).max() * np.abs(xv).sum()


@pytest.mark.parametrize("p", [2, 3, 5])
def test_invariance_under_renumbering(p):
    c0, q0 = quad_lattice(3, 0.15, seed=5)
    c1, q1 = quad_lattice(3, 0.15, seed=5, shuffle=True, shuffle_seed=17)
    P0, P1 = twod.Problem2(c0, q0, p, p + 2), twod.Problem2(c1, q1, p, p + 2)
    X0, X1 = P0.dof_coords(), P1.dof_coords()
    key = lambda X: np.lexsort(np.round(X, 12).T[::-1])
    o0, o1 = key(X0), key(X1)
    np.testing.assert_allclose(X0[o0], X1[o1], atol=1e-13)
    perm = np.empty(P0.ndof, dtype=np.int64)
    perm[o0] = o1
    np.testing.assert_allclose(P1.K.toarray()[np.ix_(perm, perm)], P0.K.toarray(), atol=1e-12)


def test_hand_numbering_p3():
    # one quad, global vertices 2 0 1 3 in local order; p = 3: 4 vertex DOFs,
    # edges 4..11 (2 each), interior 12..15.
    num = twod.numbering2(np.array([[2, 0, 1, 3]]), 3, nv=4)
    e2l = num["e2l"][0]
    L = twod.lattice2(3)
    at = lambda i1, i2: e2l[i1 + 4 * i2]
    assert at(0, 0) == 2 and at(3, 0) == 0 and at(3, 3) == 1 and at(0, 3) == 3
    # local edge 0 = global (2,0): from global 0 at (3,0) toward (0,0)
    assert at(2, 0) == 4 and at(1, 0) == 5
    # local edge 1 = global (0,1): from (3,0) toward (3,3)
    assert at(3, 1) == 6 and at(3, 2) == 7
    # local edge 2 = global (3,1): from global 1 at (3,3) toward (0,3)
    assert at(2, 3) == 8 and at(1, 3) == 9
    # local edge 3 = global (2,3): from global 2 at (0,0) toward (0,3)
    assert at(0, 1) == 10 and at(0, 2) == 11
    assert at(1, 1) == 12 and at(2, 1) == 13 and at(1, 2) == 14 and at(2, 2) == 15
    assert num["ndof"] == 16 and len(num["boundary_dofs"]) == 12


def test_stiffness_matches_the_papers_2d_setup_formula():
    """The paper's 2D diffusion setup (Sec. 5.3, the PA setup listing) stores,
    per point, c = alpha W / det J and the three symmetric entries
    c (J12^2 + J22^2), -c (J12 J11 + J22 J21), c (J11^2 + J21^2) of
    c adj(J) adj(J)^T, applied to reference gradients. The oracle's element
    stiffness (built from J^-1, J^-T and det J) must equal the stiffness
    assembled from those entries."""
    from fem_inputs import lognormal, quad_lattice
    from oracle import twod
    c, q = quad_lattice(3, 0.15, seed=12, shuffle=True)
    kap = lognormal(13, q.shape[0])
    for p in (1, 2, 4):
        ref = twod.Reference2(p, p + 2)
        X = c[q.astype(np.int64)]
        _, J, det, _ = twod.geometry2(ref, X)
        J11, J12, J21, J22 = J[..., 0, 0], J[..., 0, 1], J[..., 1, 0], J[..., 1, 1]
        cq = kap[:, None] * ref.w[None, :] / det
        Y = np.empty(J.shape)
        Y[..., 0, 0] = cq * (J12 ** 2 + J22 ** 2)
        Y[..., 0, 1] = Y[..., 1, 0] = -cq * (J12 * J11 + J22 * J21)
        Y[..., 1, 1] = cq * (J11 ** 2 + J21 ** 2)
        K_listing = np.einsum("qai,eqab,qbj->eij", ref.dphi, Y, ref.dphi, optimize=True)
        K = twod.stiffness2(ref, X, kap)
        assert np.abs(K - K_listing).max() <= 1e-13 * np.abs(K).max()
