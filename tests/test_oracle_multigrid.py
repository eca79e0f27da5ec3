"""Pins for the p-multigrid oracle (oracle.multigrid): level orders, the
hash start vector, 1D interpolation, prolongation of polynomials, the coarse
essential-DOF rule, the Chebyshev smoother against its closed-form error
polynomial, the power-iteration bound, symmetry and contraction of the
V-cycle with an exact coarse solve, and flexible CG."""

import types

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from fem_inputs import hex_lattice, lognormal, x_uniform
from oracle import assemble, multigrid as mg, numbering, rules, solve as osolve


def test_level_orders():
    assert mg.level_orders(8) == [8, 4, 2, 1]
    assert mg.level_orders(5) == [5, 2, 1]
    assert mg.level_orders(3) == [3, 1]
    assert mg.level_orders(1) == [1]


def test_start_vector_closed_form():
    v = mg.start_vector(4)
    assert v[0] == -0.5
    assert v[1] == 2654435761 / 2 ** 32 - 0.5
    assert v[2] == ((2 * 2654435761) % 2 ** 32) / 2 ** 32 - 0.5
    assert abs(v[1] - (0.5 * (np.sqrt(5) - 1) - 0.5)) < 5e-9   # 2654435761 ~ 2^32 / golden ratio


@pytest.mark.parametrize("pf,pc", [(2, 1), (4, 2), (5, 2), (8, 4), (3, 1)])
def test_interp_1d(pf, pc):
    I = mg.interp_1d(pf, pc)
    assert I.shape == (pf + 1, pc + 1)
    np.testing.assert_allclose(I.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(I[0], np.eye(pc + 1)[0], atol=1e-14)
    np.testing.assert_allclose(I[-1], np.eye(pc + 1)[-1], atol=1e-14)
    xc, xf = rules.gll_nodes(pc), rules.gll_nodes(pf)
    for k in range(pc + 1):
        np.testing.assert_allclose(I @ xc ** k, xf ** k, atol=1e-13)
    # one degree more is not reproduced
    assert np.abs(I @ xc ** (pc + 1) - xf ** (pc + 1)).max() > 1e-6


@pytest.mark.parametrize("pf,pc,shuffle", [(2, 1, False), (4, 2, True), (5, 2, True), (8, 4, False)])
def test_prolongation_reproduces_coarse_polynomials(pf, pc, shuffle):
    c, h = hex_lattice(2, 0.0, seed=1, shuffle=shuffle)      # affine elements
    f = assemble.Problem(c, h, pf, pf + 2)
    co = assemble.Problem(c, h, pc, pc + 2)
    P = mg.prolongation(f.e2l, pf, f.ndof, co.e2l, pc, co.ndof)
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-13)
    Xf, Xc = f.dof_coords(), co.dof_coords()
    for g in (lambda X: X[:, 0] ** pc * X[:, 1] - 2.0 * X[:, 2] ** pc + 0.5,
              lambda X: (X[:, 0] * X[:, 1] * X[:, 2]) ** pc + X[:, 1]):
        np.testing.assert_allclose(P @ g(Xc), g(Xf), atol=1e-12)


@pytest.mark.parametrize("p", [2, 4, 5])
def test_coarse_essential_rule(p):
    c, h = hex_lattice(3, 0.1, seed=2, shuffle=True)
    f = assemble.Problem(c, h, p, p + 2)
    co = assemble.Problem(c, h, p // 2, p // 2 + 2)
    # whole boundary -> whole coarse boundary
    m = mg.coarse_essential(f.e2l, p, f.num["boundary_mask"], co.e2l, p // 2, co.ndof)
    np.testing.assert_array_equal(m, co.num["boundary_mask"])
    # one face (x = 0) -> the coarse DOFs on that face
    Xf, Xc = f.dof_coords(), co.dof_coords()
    mf = np.abs(Xf[:, 0]) < 1e-12
    m = mg.coarse_essential(f.e2l, p, mf, co.e2l, p // 2, co.ndof)
    np.testing.assert_array_equal(m, np.abs(Xc[:, 0]) < 1e-12)
    # one face-interior fine DOF missing: exactly the (pc-1)^2 coarse
    # face-interior DOFs of that face become free, nothing else changes
    pc = p // 2
    if pc >= 2:
        L = numbering.lattice(p)
        for e in range(f.E):
            for k in range(L.shape[0]):
                i = f.e2l[e, k]
                inside = [(0 < L[k, d] < p) for d in range(3)]
                if mf[i] and sum(inside) == 2:
                    break
            else:
                continue
            break
        mf2 = mf.copy()
        mf2[i] = False
        m2 = mg.coarse_essential(f.e2l, p, mf2, co.e2l, pc, co.ndof)
        assert np.all(m2 <= m) and m.sum() - m2.sum() == (pc - 1) ** 2


def _diag_level(lams):
    n = len(lams)
    return types.SimpleNamespace(A=sp.diags(np.asarray(lams, dtype=np.float64)).tocsr(), D=np.ones(n), lam=None,
                                 ess=np.zeros(n, dtype=bool))


@pytest.mark.parametrize("K,alpha", [(1, 0.3), (2, 0.25), (3, 0.2), (5, 0.1)])
def test_chebyshev_error_polynomial(K, alpha):
    """For A = diag(lam), D = I: e - z = p_K(lam) e with
    p_K(l) = T_K((theta - l) / delta) / T_K(theta / delta)."""
    lams = np.array([0.05, 0.2, 0.4, 0.7, 1.0, 1.3, 1.6, 1.9, 2.05])
    M = mg.PMG.__new__(mg.PMG)
    M.K, M.alpha, M.beta = K, alpha, 1.1
    lv = _diag_level(lams)
    lv.lam = 1.9
    hi = 1.1 * 1.9
    lo = alpha * hi
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    T = np.polynomial.chebyshev.Chebyshev.basis(K)
    pk = T((th - lams) / de) / T(th / de)
    e = np.linspace(1.0, 2.0, lams.size)
    r = lv.A @ e
    z, res = M.smooth(lv, r)
    np.testing.assert_allclose(e - z, pk * e, atol=1e-13)
    np.testing.assert_allclose(res, r - lv.A @ z, atol=1e-13)
    # post-smoothing from z0 multiplies the error by p_K again
    z0 = 0.3 * e
    z2, _ = M.smooth(lv, r, z0.copy())
    np.testing.assert_allclose(e - z2, pk * (e - z0), atol=1e-13)


def test_power_lambda_lower_bound_and_accuracy():
    c, h = hex_lattice(3, 0.15, seed=4)
    f = assemble.Problem(c, h, 3, 5, kappa=lognormal(3, h.shape[0]))
    ess = f.num["boundary_dofs"]
    A = osolve.constrain(f.K, ess)
    D = A.diagonal()
    free = np.ones(f.ndof)
    free[ess] = 0.0
    lam = mg.power_lambda(A, D, free, 20)
    idx = np.nonzero(free)[0]
    S = (A.toarray() / np.sqrt(D)[:, None] / np.sqrt(D)[None, :])[np.ix_(idx, idx)]
    lmax = np.linalg.eigvalsh(S).max()
    assert lam <= lmax * (1 + 1e-12)
    assert lam >= 0.9 * lmax


class _ExactCoarse(mg.PMG):
    def coarse_solve(self, lv, r):
        return spla.spsolve(lv.A.tocsc(), r)


def _pmg(p=4, N=3, cls=mg.PMG, **kw):
    c, h = hex_lattice(N, 0.15, seed=6, shuffle=True)
    kap = lognormal(7, h.shape[0])
    f = assemble.Problem(c, h, p, p + 2, kappa=kap)
    ess = f.num["boundary_dofs"]
    return cls(c, h, p, p + 2, kap, ess, fine_prob=f, **kw), f, ess


@pytest.mark.parametrize("p", [2, 4])
def test_vcycle_symmetric_positive_with_exact_coarse(p):
    M, f, ess = _pmg(p, cls=_ExactCoarse)
    free = np.ones(f.ndof)
    free[ess] = 0.0
    u = x_uniform(1, f.ndof) * free
    v = x_uniform(2, f.ndof) * free
    Vu, Vv = M.vcycle(u), M.vcycle(v)
    assert abs(v @ Vu - u @ Vv) <= 1e-12 * np.abs(v).sum() * np.abs(Vu).max()
    assert u @ Vu > 0 and v @ Vv > 0
    # error propagation I - V A contracts in the A-norm
    A = M.levels[0].A
    e = u
    e2 = e - M.vcycle(A @ e)
    assert np.sqrt(e2 @ (A @ e2)) < 0.5 * np.sqrt(e @ (A @ e))


def test_fcg():
    M, f, ess = _pmg(4)
    b = osolve.constrain_rhs(f.K, x_uniform(3, f.ndof), ess)
    x, it, rel = M.fcg(b, rtol=1e-10)
    assert rel <= 1.01e-10 and it < 30
    Ac = M.levels[0].A
    xs = spla.spsolve(Ac.tocsc(), b)
    assert np.abs(x - xs).max() <= 1e-7 * np.abs(xs).max()
    # with a fixed linear SPD preconditioner (Jacobi) flexible CG is PCG:
    # the same iterates after k steps
    D = Ac.diagonal()
    M3, _, _ = _pmg(4)
    M3.vcycle = lambda r, l=0: r / D
    for k in (1, 3, 8):
        xk, itk, _ = M3.fcg(b, rtol=1e-300, maxit=k)
        xp, _ = osolve.pcg(Ac, b, rtol=1e-300, maxit=k)
        assert itk == k
        np.testing.assert_allclose(xk, xp, rtol=0, atol=1e-10 * np.abs(xp).max())
    # with an exact preconditioner FCG takes one step
    M2, _, _ = _pmg(4)
    M2.vcycle = lambda r, l=0: spla.spsolve(Ac.tocsc(), r)
    _, it2, rel2 = M2.fcg(b, rtol=1e-10)
    assert it2 == 1 and rel2 < 1e-10


def test_single_level_is_coarse_cg():
    """p = 1: the preconditioner is the fixed-count coarse PCG itself."""
    M, f, ess = _pmg(1, N=4, coarse_its=7)
    r = osolve.constrain_rhs(f.K, x_uniform(4, f.ndof), ess)
    Ac = M.levels[0].A
    x, info = osolve.pcg(Ac, r, rtol=1e-300, maxit=7)
    np.testing.assert_allclose(M.vcycle(r), x, rtol=0, atol=1e-12 * np.abs(x).max())


# ---- vector (elasticity) hierarchy
def _epmg(p=4, N=3, cls=mg.PMG, ess_kind="clamped", **kw):
    from oracle import elasticity
    c, h = hex_lattice(N, 0.15, seed=8, shuffle=True)
    E = h.shape[0]
    lam, mu = lognormal(9, E), lognormal(10, E)
    f = elasticity.ElasticityProblem(c, h, p, p + 2, lam, mu)
    bd = assemble.Problem(c, h, p, p + 2).num["boundary_dofs"]
    n = f.ndof
    if ess_kind == "clamped":
        ess = np.concatenate([bd + k * n for k in range(3)])
    elif ess_kind == "x-only":
        ess = bd
    else:
        ess = np.zeros(0, dtype=np.int64)
    return cls(c, h, p, p + 2, None, ess, fine_prob=f, lame=(lam, mu), **kw), f, ess, (c, h)


def test_vector_prolongation_reproduces_linear_fields():
    """P (no essential DOFs) maps the coarse interpolant of a linear vector
    field to the fine one, component by component."""
    M, f, _, (c, h) = _epmg(4, N=2, ess_kind="none")
    Xf = assemble.Problem(c, h, 4, 6).dof_coords()
    Xc = assemble.Problem(c, h, 2, 4).dof_coords()
    A = np.array([[0.3, -1.2, 0.5], [0.7, 0.1, -0.4], [-0.2, 0.9, 0.6]])
    t = np.array([0.25, -0.5, 1.0])
    vec = lambda X: np.concatenate([(X @ A.T + t)[:, k] for k in range(3)])
    np.testing.assert_allclose(M.levels[0].P @ vec(Xc), vec(Xf), atol=1e-12)


def test_vector_coarse_essential_per_component():
    M, f, ess, (c, h) = _epmg(4, N=2, ess_kind="x-only")
    co = assemble.Problem(c, h, 2, 4)
    m = M.levels[1].ess
    nc = co.ndof
    # component 0: the coarse boundary; components 1, 2: nothing
    assert set(np.nonzero(m[:nc])[0]) == set(co.num["boundary_dofs"])
    assert not m[nc:].any()
    M2, _, _, _ = _epmg(4, N=2, ess_kind="clamped")
    assert M2.levels[1].ess.sum() == 3 * len(co.num["boundary_dofs"])


def test_vector_vcycle_and_fcg():
    """Symmetric positive V-cycle with an exact coarse solve that contracts
    the A-norm error; flexible CG reaches the Cholesky solution in far fewer
    iterations than Jacobi-PCG."""
    M, f, ess, _ = _epmg(4, cls=_ExactCoarse)
    n = M.levels[0].n
    free = np.ones(n)
    free[ess] = 0.0
    u = x_uniform(11, n) * free
    v = x_uniform(12, n) * free
    Vu, Vv = M.vcycle(u), M.vcycle(v)
    assert abs(v @ Vu - u @ Vv) <= 1e-12 * np.abs(v).sum() * np.abs(Vu).max()
    assert u @ Vu > 0 and v @ Vv > 0
    A = M.levels[0].A
    e2 = u - M.vcycle(A @ u)
    assert np.sqrt(e2 @ (A @ e2)) < 0.5 * np.sqrt(u @ (A @ u))
    M1, f, ess, _ = _epmg(4)
    b = osolve.constrain_rhs(f.K, x_uniform(13, n), ess)
    x, it, rel = M1.fcg(b, rtol=1e-10)
    xs = spla.spsolve(A.tocsc(), b)
    assert rel <= 1.01e-10 and np.abs(x - xs).max() <= 1e-7 * np.abs(xs).max()
    _, info = osolve.pcg(A, b, rtol=1e-10)
    assert it < 40 and 3 * it < info["iterations"]
